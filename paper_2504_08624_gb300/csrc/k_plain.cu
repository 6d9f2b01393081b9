// Plain sequential-per-channel path: the comparison baseline for the scan and
// fused kernels.  It mirrors running one library op per filter of a TorchFX
// chain (Sec. 3 pipe operator; Sec. 4 Tables 2-4): one kernel per stage, the
// IIR walked sample by sample by one thread per channel, the FIR summed
// directly by one thread per output sample.
#include "tfx_common.cuh"

namespace tfx {

// One thread per channel; the whole cascade is advanced one sample at a time,
// each section as the same 2-state recursion the scan kernel uses.
// coef rows: b0 c1 c2 a1 a2 (+3 pad), c1 = b1 - a1 b0, c2 = b2 - a2 b0.
__global__ void k_plain_sos(const float* __restrict__ x, float* __restrict__ y, int64_t C, int64_t N,
                            int64_t ldx, int64_t ldy, int S, const float* __restrict__ coef) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    constexpr int SMAX = 64;
    float w1[SMAX], w2[SMAX];
    for (int s = 0; s < S; ++s) w1[s] = w2[s] = 0.f;
    const float* xr = x + c * ldx;
    float* yr = y + c * ldy;
    for (int64_t n = 0; n < N; ++n) {
        float v = xr[n];
        for (int s = 0; s < S; ++s) {
            const float* cf = coef + 8 * s;
            const float yv = fmaf(cf[0], v, w1[s]);
            const float n1 = fmaf(cf[1], v, fmaf(-cf[3], w1[s], w2[s]));
            w2[s] = fmaf(cf[2], v, -cf[4] * w1[s]);
            w1[s] = n1;
            v = yv;
        }
        yr[n] = v;
    }
}

// One thread per output sample, direct causal sum.
__global__ void k_plain_fir(const float* __restrict__ x, float* __restrict__ y, int64_t C, int64_t N,
                            int64_t ldx, int64_t ldy, int L, const float* __restrict__ h) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= C * N) return;
    const int64_t c = idx / N, n = idx % N;
    const float* xr = x + c * ldx;
    const int64_t kmax = n < (int64_t)L - 1 ? n : (int64_t)L - 1;
    float acc = 0.f;
    for (int64_t k = 0; k <= kmax; ++k) acc = fmaf(h[k], xr[n - k], acc);
    y[c * ldy + n] = acc;
}

__global__ void k_copy_rows(const float* __restrict__ x, float* __restrict__ y, int64_t C, int64_t N,
                            int64_t ldx, int64_t ldy) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= C * N) return;
    const int64_t c = idx / N, n = idx % N;
    y[c * ldy + n] = x[c * ldx + n];
}

cudaError_t launch_plain_sos(const float* x, float* y, int64_t C, int64_t N, int64_t ldx, int64_t ldy,
                             int S, const float* coef, cudaStream_t s) {
    if (C <= 0 || N <= 0) return cudaSuccess;
    if (S > 64) return cudaErrorInvalidValue;
    const int bs = 64;
    k_plain_sos<<<(unsigned)((C + bs - 1) / bs), bs, 0, s>>>(x, y, C, N, ldx, ldy, S, coef);
    return cudaGetLastError();
}

cudaError_t launch_plain_fir(const float* x, float* y, int64_t C, int64_t N, int64_t ldx, int64_t ldy,
                             int L, const float* taps, cudaStream_t s) {
    if (C <= 0 || N <= 0) return cudaSuccess;
    const int bs = 256;
    const int64_t n = C * N;
    k_plain_fir<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(x, y, C, N, ldx, ldy, L, taps);
    return cudaGetLastError();
}

cudaError_t launch_copy_rows(const float* x, float* y, int64_t C, int64_t N, int64_t ldx, int64_t ldy,
                             cudaStream_t s) {
    if (C <= 0 || N <= 0) return cudaSuccess;
    const int bs = 256;
    const int64_t n = C * N;
    k_copy_rows<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(x, y, C, N, ldx, ldy);
    return cudaGetLastError();
}

}  // namespace tfx
