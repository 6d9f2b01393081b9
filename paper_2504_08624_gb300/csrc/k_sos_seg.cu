// Segment start fix-up for cascades run by channel segments (the
// tensor-core block-state kernel, k_sos_tc.cu).
//
// A segment other than a channel's first is run from zero state; its true
// start state s differs, and by linearity the output differs exactly by the
// cascade's free response from s, y_free[n] = C A^n s (A the one-sample
// transfer of the 2S-dimensional cascade state, C its output row).  The
// segment kernel records each segment's zero-start end state e_k;
// k_sos_seg_fix chains the true start states s_(k+1) = A^Lseg s_k + e_k and
// adds y_free over the first D samples of every segment, where the plan chose
// D (from the powers of A in FP64) so that the free response beyond D is below
// 1e-9 of its initial size.
#include "sos_pass.cuh"

namespace tfx {
namespace {

constexpr int SEG_WARPS = 4;

// y[n] += free response of the true start state, first D samples of every
// segment k >= 1.  One warp per (segment, round of 2048 samples); lane l
// handles the 64-sample chunk j = 32 round + l, whose start state A^(64 j) s
// is formed from the binary powers A^(64 * 2^k) (the same matrix for every
// lane at each step).  The true start state chains back J segments
// (s_k = A^Lseg s_(k-1) + e_(k-1); the plan picked J so that A^(J Lseg) is
// negligible).
__global__ void __launch_bounds__(32 * SEG_WARPS) k_sos_seg_fix(SegArgs a) {
    constexpr int NS = 2 * SEG_SMAX;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rounds = (a.D + 2047) / 2048;
    const int64_t nfix = a.C * (a.P - 1) * rounds;
    const int64_t g = (int64_t)blockIdx.x * SEG_WARPS + warp;
    if (g >= nfix) return;
    const int64_t round = g % rounds, seg = g / rounds;
    const int64_t c = seg / (a.P - 1), k = seg % (a.P - 1) + 1;
    const int S = a.S, n2 = 2 * S;
    // true start state of segment k (lane r < 2S holds s[r])
    float sr = 0.f;
    for (int64_t j = k - a.J < 0 ? 0 : k - a.J; j < k; ++j) {
        const float2 ej = lane < n2 ? a.e_out[(c * a.P + j) * SEG_SMAX + (lane >> 1)] : make_float2(0.f, 0.f);
        float acc = (lane & 1) ? ej.y : ej.x;
#pragma unroll
        for (int m = 0; m < NS; ++m) {
            const float sm = __shfl_sync(0xffffffffu, sr, m);
            if (lane < n2 && m < n2) acc = fmaf(a.Phi[lane * 16 + m], sm, acc);
        }
        sr = acc;
    }
    // every lane takes the whole start state before any lane leaves
    float w[NS];
#pragma unroll
    for (int m = 0; m < NS; ++m) w[m] = __shfl_sync(0xffffffffu, sr, m);
    const int64_t chunk = round * 32 + lane;
    const int o0 = (int)(chunk * 64);  // offset of the chunk within the segment
    const int64_t seg0 = k * a.Lseg;
    if (o0 >= a.D || seg0 + o0 >= a.N) return;  // no shuffles below
    // chunk start state w = A^(64 chunk) s
    for (int b = 0; b < SEG_NPOW; ++b) {
        if (!((chunk >> b) & 1)) continue;
        const float* Pm = a.Pk + (size_t)b * 256;
        float nw[NS];
#pragma unroll
        for (int r = 0; r < NS; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int m = 0; m < NS; ++m)
                if (r < n2 && m < n2) acc = fmaf(Pm[r * 16 + m], w[m], acc);
            nw[r] = acc;
        }
#pragma unroll
        for (int r = 0; r < NS; ++r) w[r] = nw[r];
    }
    float cb0[SEG_SMAX], cc1[SEG_SMAX], cc2[SEG_SMAX], ca1[SEG_SMAX], ca2[SEG_SMAX];
#pragma unroll
    for (int i = 0; i < SEG_SMAX; ++i) {
        const bool on = i < S;
        cb0[i] = on ? a.coef[8 * i + 0] : 0.f;
        cc1[i] = on ? a.coef[8 * i + 1] : 0.f;
        cc2[i] = on ? a.coef[8 * i + 2] : 0.f;
        ca1[i] = on ? a.coef[8 * i + 3] : 0.f;
        ca2[i] = on ? a.coef[8 * i + 4] : 0.f;
    }
    // free response over the chunk, in registers
    float yf[64];
#pragma unroll
    for (int t = 0; t < 64; ++t) {
        float v = 0.f;  // zero input: each section driven by the previous one's free output
#pragma unroll
        for (int i = 0; i < SEG_SMAX; ++i) {
            if (i < S) {
                const float w1 = w[2 * i], w2 = w[2 * i + 1];
                const float y = fmaf(cb0[i], v, w1);
                w[2 * i] = fmaf(cc1[i], v, fmaf(-ca1[i], w1, w2));
                w[2 * i + 1] = fmaf(cc2[i], v, -ca2[i] * w1);
                v = y;
            }
        }
        yf[t] = a.gain * v;
    }
    const int64_t n0 = seg0 + o0;
    int64_t lim = a.N - n0 < 64 ? a.N - n0 : 64;  // the chunk lies inside the segment (D <= Lseg)
    if (a.D - o0 < lim) lim = a.D - o0;
    float* p = a.y + c * a.ldy + n0;
    if (lim == 64 && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
        float4* p4 = reinterpret_cast<float4*>(p);
        float4 cur[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) cur[q] = p4[q];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            p4[q] = make_float4(cur[q].x + yf[4 * q], cur[q].y + yf[4 * q + 1], cur[q].z + yf[4 * q + 2],
                                cur[q].w + yf[4 * q + 3]);
    } else {
#pragma unroll
        for (int t = 0; t < 64; ++t)
            if (t < lim) p[t] += yf[t];
    }
}

}  // namespace

cudaError_t launch_seg_fix(const SegArgs& a, cudaStream_t s) {
    if (a.C <= 0 || a.N <= 0 || a.P <= 1 || a.D <= 0) return cudaSuccess;
    const int64_t fixes = a.C * (a.P - 1) * ((a.D + 2047) / 2048);
    k_sos_seg_fix<<<(unsigned)((fixes + SEG_WARPS - 1) / SEG_WARPS), 32 * SEG_WARPS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tfx
