// Measurement helper: the FP32 fused multiply-add throughput of this GPU, the
// denominator of the CUDA-core rooflines (the scan kernels and the FFT
// butterflies are FP32 arithmetic).  Each thread runs 8 independent FMA
// chains (scalar fmaf, or the packed two-lane form), so the issue slots, not
// the FMA latency, set the rate when enough warps are resident.
#include "tfx_common.cuh"
#include "tfx.h"

namespace tfx {
namespace {

constexpr int PROBE_CHAINS = 8;

__global__ void k_fma_probe(float* out, int iters, float a, float b) {
    float v[PROBE_CHAINS];
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) v[j] = (float)(threadIdx.x + j) * 1e-3f;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) v[j] = fmaf(v[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) s += v[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_fma2_probe(float* out, int iters, float a, float b) {
    float2 v[PROBE_CHAINS];
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) v[j] = make_float2((float)(threadIdx.x + j) * 1e-3f, (float)j);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) v[j] = __ffma2_rn(v[j], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) s += v[j].x + v[j].y;
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace tfx

extern "C" int tfx_fma_probe(float* out, int32_t blocks, int32_t threads, int32_t iters, int32_t packed,
                             tfx_stream s) {
    if (!out || blocks <= 0 || threads <= 0 || threads > 1024 || threads % 32 != 0 || iters <= 0)
        return TFX_ERR_INVALID;
    // a and b keep every chain bounded: v -> 0.999 v + 1e-4 converges to 0.1
    if (packed)
        tfx::k_fma2_probe<<<blocks, threads, 0, (cudaStream_t)s>>>(out, iters, 0.999f, 1e-4f);
    else
        tfx::k_fma_probe<<<blocks, threads, 0, (cudaStream_t)s>>>(out, iters, 0.999f, 1e-4f);
    return cudaGetLastError() == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
}

extern "C" double tfx_fma_probe_flops(int32_t blocks, int32_t threads, int32_t iters, int32_t packed) {
    return 2.0 * (packed ? 2.0 : 1.0) * tfx::PROBE_CHAINS * (double)blocks * threads * iters;
}
