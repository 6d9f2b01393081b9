// Per-thread pieces of the block-tile SOS cascade scan (k_unit): chunk loads
// and stores, and one section's pass over a thread's chunk fused with the
// previous section's fix-up.
#pragma once

#include "tfx_common.cuh"

namespace tfx {

template <int T>
__device__ __forceinline__ void load_chunk(const float* row, int64_t n0, int64_t N, float (&u)[T]) {
    const float* p = row + n0;
    if (n0 + T <= N && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
        const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < T / 4; ++i) {
            float4 v = p4[i];
            u[4 * i + 0] = v.x;
            u[4 * i + 1] = v.y;
            u[4 * i + 2] = v.z;
            u[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < T; ++i) u[i] = (n0 + i < N) ? p[i] : 0.f;
    }
}

template <int T>
__device__ __forceinline__ void store_chunk(float* row, int64_t n0, int64_t N, const float (&u)[T], float g) {
    float* p = row + n0;
    if (n0 + T <= N && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
        float4* p4 = reinterpret_cast<float4*>(p);
#pragma unroll
        for (int i = 0; i < T / 4; ++i)
            p4[i] = make_float4(u[4 * i] * g, u[4 * i + 1] * g, u[4 * i + 2] * g, u[4 * i + 3] * g);
    } else {
#pragma unroll
        for (int i = 0; i < T; ++i)
            if (n0 + i < N) p[i] = u[i] * g;
    }
}

// One step of a cascade scan over a thread's chunk u[0, T): the fix-up of
// section s-1 (`fix`: add its homogeneous response yh[t] = -pa1 yh[t-1] -
// pa2 yh[t-2] from its true chunk-start state st) fused with the zero-state
// pass of section s (`run`), whose transposed-direct-form-II state (w1, w2)
// is updated as w1' = c1 v - a1 w1 + w2, w2' = c2 v - a2 w1, y = b0 v + w1
// (c1 = b1 - a1 b0, c2 = b2 - a2 b0 formed in FP64 at plan time).  On return
// (w1, w2) is the chunk's zero-state end state of section s.  Three loop
// bodies, so that no predicated-off instruction is issued.
template <int T>
__device__ __forceinline__ void section_pass(float (&u)[T], bool fix, bool run, float b0, float c1, float c2,
                                             float a1, float a2, float2 st, float pa1, float pa2, float& w1,
                                             float& w2) {
    w1 = 0.f;
    w2 = 0.f;
    if (run && !fix) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float v = u[t];
            u[t] = fmaf(b0, v, w1);
            const float n1 = fmaf(c1, v, fmaf(-a1, w1, w2));
            w2 = fmaf(c2, v, -a2 * w1);
            w1 = n1;
        }
    } else if (run) {
        float h1 = st.x, h2 = 0.f;
        {
            const float v = u[0] + st.x;
            u[0] = fmaf(b0, v, w1);
            const float n1 = fmaf(c1, v, fmaf(-a1, w1, w2));
            w2 = fmaf(c2, v, -a2 * w1);
            w1 = n1;
        }
        {
            const float h = fmaf(-pa1, h1, st.y);
            h2 = h1;
            h1 = h;
            const float v = u[1] + h;
            u[1] = fmaf(b0, v, w1);
            const float n1 = fmaf(c1, v, fmaf(-a1, w1, w2));
            w2 = fmaf(c2, v, -a2 * w1);
            w1 = n1;
        }
#pragma unroll
        for (int t = 2; t < T; ++t) {
            const float h = fmaf(-pa1, h1, -pa2 * h2);
            h2 = h1;
            h1 = h;
            const float v = u[t] + h;
            u[t] = fmaf(b0, v, w1);
            const float n1 = fmaf(c1, v, fmaf(-a1, w1, w2));
            w2 = fmaf(c2, v, -a2 * w1);
            w1 = n1;
        }
    } else if (fix) {
        float h1 = st.x, h2 = 0.f;
        u[0] += st.x;
        {
            const float h = fmaf(-pa1, h1, st.y);
            h2 = h1;
            h1 = h;
            u[1] += h;
        }
#pragma unroll
        for (int t = 2; t < T; ++t) {
            const float h = fmaf(-pa1, h1, -pa2 * h2);
            h2 = h1;
            h1 = h;
            u[t] += h;
        }
    }
}

}  // namespace tfx
