// Device helpers shared by the tensor-core kernels: FP32 -> 16-bit hi/lo
// operand splitting, guarded 8-sample loads, bounded mbarrier waits and named
// barriers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_ptx.cuh"
#include "tfx_common.cuh"

namespace tfx {

// Split 8 consecutive samples into hi / lo parts packed as 16-byte chunks:
// BF16 hi + BF16 lo, or (after scaling by an exact power of two) FP16 hi +
// FP16 lo.  The low part is the rounded residual v - hi, which is exact in FP32.
__device__ __forceinline__ void split8_bf16(const float (&v)[8], uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * i]);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(v[2 * i + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * i] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * i + 1] - __bfloat162float(h1));
        h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void split8_f16(const float (&v)[8], float scale, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // pairs by the packed conversions (same roundings)
        const float s0 = v[2 * i] * scale, s1 = v[2 * i + 1] * scale;
        const __half2 hh = __floats2half2_rn(s0, s1);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(s0 - hf.x, s1 - hf.y);
        h[i] = *reinterpret_cast<const uint32_t*>(&hh);
        l[i] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// 8 consecutive samples starting at t (zero outside [0, N)).
__device__ __forceinline__ void load8(const float* xr, int64_t t, int64_t N, bool vec, float (&v)[8]) {
    if (vec && t >= 0 && t + 8 <= N) {
        const float4 p0 = *reinterpret_cast<const float4*>(xr + t);
        const float4 p1 = *reinterpret_cast<const float4*>(xr + t + 4);
        v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w;
        v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (t + i >= 0 && t + i < N) ? xr[t + i] : 0.f;
    }
}

// 8 consecutive samples starting at t as one 32-byte load when the address is
// 32-byte aligned (vec32) and the chunk lies inside [0, N); otherwise load8.
// The samples are read once: the load does not allocate in L1, which is small
// beside a kernel's large shared-memory carve-out (measured: the tensor-core
// cascade 0.543 -> 0.493 ms).
__device__ __forceinline__ void load8_32(const float* xr, int64_t t, int64_t N, bool vec32, bool vec,
                                         float (&v)[8]) {
    if (vec32 && t >= 0 && t + 8 <= N) {
        asm volatile("ld.global.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                     : "l"(xr + t));
    } else {
        load8(xr, t, N, vec, v);
    }
}

// Bounded wait on an mbarrier phase: false (and the status word set) once the
// time limit passes or another CTA has already recorded an error.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, int* status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*(volatile int*)status != 0) return false;
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            atomicCAS(status, 0, (int)TFX_ERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

}  // namespace tfx
