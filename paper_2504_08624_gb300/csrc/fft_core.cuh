// Register-resident FFT building blocks shared by the overlap-save FIR
// kernels (k_fir_fft.cu) and the spectral training kernels (k_spectral.cu):
// the radix-16 passes, the shared-memory exchanges between them, and the
// loads and stores of two real segments as one complex sequence.  The
// algorithm and the data layouts are described at the top of k_fir_fft.cu.
#pragma once

#include "tfx_common.cuh"

namespace tfx {
namespace {

// Complex sum and difference as one packed two-lane FP32 instruction each
// (the real and imaginary parts are the two lanes; each lane rounds as the
// scalar instruction does).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 ra, rb, rr;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rr, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rr;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 ra, rb, rr;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rr, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rr;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// cos(2 pi k / 32), k = 0..8 (FP32): the constant twiddles of the in-register
// DFTs of up to 32 points are these and their negatives.
__device__ __forceinline__ constexpr float cos32(int k) {
    return k == 0 ? 1.0f
         : k == 1 ? 0.98078528040323043f
         : k == 2 ? 0.92387953251128674f
         : k == 3 ? 0.83146961230254524f
         : k == 4 ? 0.70710678118654752f
         : k == 5 ? 0.55557023301960218f
         : k == 6 ? 0.38268343236508978f
         : k == 7 ? 0.19509032201612826f
                  : 0.0f;
}

// v * e^(-2 pi i P / N) (INV: e^(+2 pi i P / N)) for the constant twiddles of
// the in-register DFT (N <= 32, P < N/2): exact for P = 0 and a quarter turn.
template <int P, int N, bool INV>
__device__ __forceinline__ float2 twc(float2 v) {
    constexpr int Q = (32 / N) * P;  // thirty-seconds of a turn, 0..15
    if constexpr (Q == 0) {
        return v;
    } else if constexpr (Q == 8) {
        return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else {
        // cos and sin of 2 pi Q / 32
        constexpr float c = Q < 8 ? cos32(Q) : -cos32(16 - Q);
        constexpr float s = Q < 8 ? cos32(8 - Q) : cos32(Q - 8);
        return INV ? make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.y, c, v.x * s))
                   : make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -v.x * s));
    }
}

// One radix-2 stage (half-distance H) of the G-point DFT over registers
// v[OFF + q*ST], q < G; butterflies q = Q, Q+1, ... by recursion.  Sums and
// differences are packed two-lane instructions; a quarter-turn twiddle
// (multiplication by -i or +i, which swaps the lanes) is folded into scalar
// sums and differences instead.
template <int G, int ST, int OFF, int H, bool INV, int Q = 0, int NV>
__device__ __forceinline__ void stage(float2 (&v)[NV]) {
    if constexpr (Q < G) {
        if constexpr ((Q / H) % 2 == 0) {
            constexpr int i0 = OFF + Q * ST, i1 = OFF + (Q + H) * ST;
            constexpr int T32 = (32 / (2 * H)) * (Q % H);  // twiddle in thirty-seconds of a turn
            const float2 a = v[i0];
            const float2 c = v[i1];
            if constexpr (T32 == 0) {
                v[i0] = cadd(a, c);
                v[i1] = csub(a, c);
            } else if constexpr (T32 == 8) {
                if constexpr (!INV) {  // DIF: (a + c, (a - c)(-i))
                    v[i0] = cadd(a, c);
                    v[i1] = make_float2(a.y - c.y, c.x - a.x);
                } else {  // DIT: (a + c i, a - c i)
                    v[i0] = make_float2(a.x - c.y, a.y + c.x);
                    v[i1] = make_float2(a.x + c.y, a.y - c.x);
                }
            } else if constexpr (!INV) {  // DIF: (a, c) -> (a + c, (a - c) w)
                v[i0] = cadd(a, c);
                v[i1] = twc<Q % H, 2 * H, false>(csub(a, c));
            } else {  // DIT: (a, c) -> (a + c w*, a - c w*)
                const float2 cw = twc<Q % H, 2 * H, true>(c);
                v[i0] = cadd(a, cw);
                v[i1] = csub(a, cw);
            }
        }
        stage<G, ST, OFF, H, INV, Q + 1>(v);
    }
}

// G-point DFT (G <= 32).  DIF: natural order in, slot q holds output
// bitrev(q).  DIT (inverse, unnormalised): bit-reversed in, natural out.
template <int G, int ST, int OFF, int NV>
__device__ __forceinline__ void dft_dif(float2 (&v)[NV]) {
    if constexpr (G >= 32) stage<G, ST, OFF, 16, false>(v);
    if constexpr (G >= 16) stage<G, ST, OFF, 8, false>(v);
    if constexpr (G >= 8) stage<G, ST, OFF, 4, false>(v);
    if constexpr (G >= 4) stage<G, ST, OFF, 2, false>(v);
    if constexpr (G >= 2) stage<G, ST, OFF, 1, false>(v);
}

template <int G, int ST, int OFF, int NV>
__device__ __forceinline__ void dft_dit(float2 (&v)[NV]) {
    if constexpr (G >= 2) stage<G, ST, OFF, 1, true>(v);
    if constexpr (G >= 4) stage<G, ST, OFF, 2, true>(v);
    if constexpr (G >= 8) stage<G, ST, OFF, 4, true>(v);
    if constexpr (G >= 16) stage<G, ST, OFF, 8, true>(v);
    if constexpr (G >= 32) stage<G, ST, OFF, 16, true>(v);
}

// A table entry by an ordinary global load, kept in program order: read-only
// (non-coherent) loads may be hoisted across the passes' barriers, and the
// kernel then holds later passes' twiddles (and the inverse's) in registers
// through the earlier ones.
__device__ __forceinline__ float2 ld_tw(const float2* p) {
    float2 r;
    asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ float4 ld_tw4(const float4* p) {
    float4 r;
    asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}

// Multiply slot q (q = Q..G-1) of the group v[OFF + q*ST] by the pass
// twiddle w_S^(i * bitrev(q)) (INV: its conjugate), read from the pass's
// table tp (row length `sub`): the twiddles of slots 2k + 1 and 2k + 2 are
// interleaved as one float4 per group position i at float4 index k*sub + i
// (one 16-byte load for two slots; consecutive i are consecutive words), and
// the last slot of an odd count is a plain row of float2 after the pairs.
template <int G, int ST, int OFF, bool INV, int Q = 1, int NV>
__device__ __forceinline__ void twiddle_group(float2 (&v)[NV], const float2* __restrict__ tp, int i, int sub) {
    if constexpr (Q < G) {
        constexpr int j0 = OFF + Q * ST;
        if constexpr (Q + 1 < G) {
            constexpr int j1 = OFF + (Q + 1) * ST;
            const float4 w = ld_tw4(reinterpret_cast<const float4*>(tp) + ((Q - 1) / 2) * sub + i);
            v[j0] = INV ? cmulc(v[j0], make_float2(w.x, w.y)) : cmul(v[j0], make_float2(w.x, w.y));
            v[j1] = INV ? cmulc(v[j1], make_float2(w.z, w.w)) : cmul(v[j1], make_float2(w.z, w.w));
            twiddle_group<G, ST, OFF, INV, Q + 2>(v, tp, i, sub);
        } else {
            const float2 w = ld_tw(tp + 2 * ((G - 1) / 2) * sub + i);
            v[j0] = INV ? cmulc(v[j0], w) : cmul(v[j0], w);
        }
    }
}

// Padded shared-memory index: one float2 of padding per 16.
__device__ __forceinline__ int pad(int n) { return n + (n >> 4); }

// Shape of the M = 2^m point transform.  PT = 16 points per thread (T = M/16
// threads): a first pass of radix G0 = 2^(m mod 4) (radix 16 when m is a
// multiple of 4), then radix-16 passes.  PT = 32 (m = 14: 512 threads):
// passes of radix 32 over spans M and M/32, then radix 16 over span 16, each
// thread holding two 16-point groups; one shared-memory exchange fewer than
// four passes need, and the second one stays within half-warps.
template <int LOGM>
struct FftShape {
    static constexpr int M = 1 << LOGM;
    static constexpr int PT = fft_pt(LOGM);
    static_assert(PT == 16 || LOGM == 14, "32 points per thread: 16384-point transforms only");
    static constexpr int T = M / PT;
    // CTAs per SM the launch bounds ask for: 1024 threads at 64 registers,
    // or one 512-thread CTA of up to 128 registers (32 complex points each)
    static constexpr int MINB = PT == 32 ? 1 : 16384 >> LOGM;
    static constexpr int R0 = PT == 16 ? LOGM % 4 : 0;  // first pass radix 2^R0 (0: radix PT)
    static constexpr int G0 = R0 ? 1 << R0 : PT;
    static constexpr int NP = PT == 32 ? 3 : (R0 ? 1 + LOGM / 4 : LOGM / 4);  // passes
    static constexpr int span(int p) {
        return PT == 32 ? (p == 0 ? M : p == 1 ? M / 32 : 16) : (p == 0 ? M : (M / G0) >> (4 * (p - 1)));
    }
    static constexpr int radix(int p) { return PT == 32 ? (p < 2 ? 32 : 16) : (p == 0 ? G0 : 16); }
    static constexpr int sub(int p) { return span(p) / radix(p); }
    // offset of pass p's twiddle table ((radix - 1) rows of `sub` entries;
    // passes with sub = 1 have none)
    static constexpr int tw_off(int p) {
        int o = 0;
        for (int q = 0; q < p; ++q)
            if (sub(q) > 1) o += (radix(q) - 1) * sub(q);
        return o;
    }
    // padded shared-memory index: one float2 per 16 (PT = 16) or per 32
    __host__ __device__ static constexpr int pad(int n) { return PT == 32 ? n + (n >> 5) : n + (n >> 4); }
};

// Padded shared-memory position of register j of thread t in pass P, as
// base(t) + off(j).  PT = 16: pass 0 (span M): point t + T*j.  A radix-16
// pass over span S (sub = S/16, which is 256, 16 or 1): point
// (t / sub) * S + t % sub + j * sub; with sub a multiple of 16 the padding
// adds j * sub/16, and with sub = 1 the point is 16t + j, padded 17t + j.
// PT = 32 (padding one per 32): pass 0: point t + 512 j, padded
// pad(t) + 528 j; pass 1 (span 512, sub 16): point (t/16) * 512 + t%16 +
// 16 j, padded base + 16 j + j/2 (t%16 < 16); pass 2 (span 16, two groups):
// point 32t + j, padded 33t + j.  In each pattern the 16 lanes of a
// half-warp touch 16 consecutive float2 (or a stride of 17 or 33): no bank
// conflicts.
template <int LOGM, int P>
struct Layout {
    using F = FftShape<LOGM>;
    static constexpr int S = F::span(P), SUB = P == 0 ? F::T : F::sub(P);
    static_assert(SUB == 1 || SUB % 16 == 0, "pass layout");
    static constexpr int STRIDE = SUB == 1 ? 1 : SUB + SUB / (F::PT == 32 ? 32 : 16);
    static constexpr int off(int j) {
        return (F::PT == 32 && SUB == 16) ? 16 * j + j / 2 : j * STRIDE;
    }
    __device__ static __forceinline__ int base(int t) {
        if constexpr (P == 0) {
            return F::pad(t);
        } else if constexpr (SUB == 1) {
            return (F::PT + 1) * t;
        } else {
            return F::pad((t / SUB) * S + t % SUB);
        }
    }
};

// First pass when G0 < 16: groups c < 16/G0, slot q of group c in register
// c + q*(16/G0), group position i = t + T*c.
template <int LOGM, bool INV, int C = 0>
__device__ __forceinline__ void first_groups(float2 (&v)[16], const float2* __restrict__ tw, int t) {
    using F = FftShape<LOGM>;
    constexpr int G = F::G0, NG = 16 / G, sub = F::M / G;
    if constexpr (C < NG) {
        const int i = t + F::T * C;
        if constexpr (!INV) {
            dft_dif<G, NG, C>(v);
            twiddle_group<G, NG, C, false>(v, tw, i, sub);
        } else {
            twiddle_group<G, NG, C, true>(v, tw, i, sub);
            dft_dit<G, NG, C>(v);
        }
        first_groups<LOGM, INV, C + 1>(v, tw, t);
    }
}

template <int LOGM, int P, bool INV>
__device__ __forceinline__ void run_pass(float2 (&v)[FftShape<LOGM>::PT], const float2* __restrict__ tw, int t) {
    using F = FftShape<LOGM>;
    if constexpr (F::PT == 16 && P == 0 && F::R0 != 0) {
        first_groups<LOGM, INV>(v, tw + F::tw_off(0), t);
    } else if constexpr (F::radix(P) < F::PT) {
        // 32 points per thread, last pass (span 16): groups in registers
        // 0..15 and 16..31, no twiddles
        static_assert(F::radix(P) == 16 && F::sub(P) == 1, "two 16-point groups");
        if constexpr (!INV) {
            dft_dif<16, 1, 0>(v);
            dft_dif<16, 1, 16>(v);
        } else {
            dft_dit<16, 1, 0>(v);
            dft_dit<16, 1, 16>(v);
        }
    } else {
        constexpr int R = F::radix(P), sub = F::sub(P);
        const float2* tp = tw + F::tw_off(P);
        const int i = t % sub;
        if constexpr (!INV) {
            dft_dif<R, 1, 0>(v);
            if constexpr (sub > 1) twiddle_group<R, 1, 0, false>(v, tp, i, sub);
        } else {
            if constexpr (sub > 1) twiddle_group<R, 1, 0, true>(v, tp, i, sub);
            dft_dit<R, 1, 0>(v);
        }
    }
}

// Threads that exchange points between pass p and pass p + 1 (either way):
// those of one span block of pass p, a contiguous run of span(p) / PT
// threads (all of them after the first pass).
template <int LOGM>
constexpr int xgroup(int p) {
    return p == 0 ? FftShape<LOGM>::T : FftShape<LOGM>::span(p) / FftShape<LOGM>::PT;
}

// Barrier over the G-thread group of thread t: the whole CTA, a warp, or a
// named barrier per group (ids 1..T/G).
template <int LOGM, int G>
__device__ __forceinline__ void group_sync(int t) {
    if constexpr (G >= FftShape<LOGM>::T) {
        __syncthreads();
    } else if constexpr (G <= 32) {
        __syncwarp();
    } else {
        static_assert(FftShape<LOGM>::T / G <= 15, "named barrier ids");
        asm volatile("bar.sync %0, %1;" ::"r"(1 + t / G), "r"(G) : "memory");
    }
}

// Move the points from pass P's layout to pass Q's (Q = P +- 1) through
// shared memory.  Only the threads of one span block of the wider pass take
// part, so the barrier between the writes and the reads is over that group;
// before the writes, every thread that may still be reading the same words
// from the previous exchange (group size PREVG, 0: none) must be done, so the
// barrier there covers the wider of the two groups.
template <int LOGM, int P, int Q, int PREVG>
__device__ __forceinline__ void exchange(float2 (&v)[FftShape<LOGM>::PT], float2* sb, int t) {
    constexpr int G = xgroup<LOGM>(P < Q ? P : Q);
    constexpr int PRE = PREVG > G ? PREVG : G;
    if constexpr (PREVG > 0) group_sync<LOGM, PRE>(t);
    float2* w = sb + Layout<LOGM, P>::base(t);
#pragma unroll
    for (int j = 0; j < FftShape<LOGM>::PT; ++j) w[Layout<LOGM, P>::off(j)] = v[j];
    group_sync<LOGM, G>(t);
    const float2* r = sb + Layout<LOGM, Q>::base(t);
#pragma unroll
    for (int j = 0; j < FftShape<LOGM>::PT; ++j) v[j] = r[Layout<LOGM, Q>::off(j)];
}

// Forward passes P.. and inverse passes ..0; PREVG is the group of the
// exchange before (0: none).  Returns nothing; the exchange group sizes are
// compile-time, so the barriers cost only what the data movement requires.
template <int LOGM, int P, int PREVG = 0>
__device__ __forceinline__ void forward_from(float2 (&v)[FftShape<LOGM>::PT], const float2* __restrict__ tw,
                                             float2* sb, int t) {
    run_pass<LOGM, P, false>(v, tw, t);
    if constexpr (P + 1 < FftShape<LOGM>::NP) {
        exchange<LOGM, P, P + 1, PREVG>(v, sb, t);
        forward_from<LOGM, P + 1, xgroup<LOGM>(P)>(v, tw, sb, t);
    }
}

template <int LOGM, int P, int PREVG = 0>
__device__ __forceinline__ void inverse_from(float2 (&v)[FftShape<LOGM>::PT], const float2* __restrict__ tw,
                                             float2* sb, int t) {
    run_pass<LOGM, P, true>(v, tw, t);
    if constexpr (P > 0) {
        exchange<LOGM, P, P - 1, PREVG>(v, sb, t);
        inverse_from<LOGM, P - 1, xgroup<LOGM>(P - 1)>(v, tw, sb, t);
    }
}

// Group size of the last exchange of a forward transform (0: none), the
// PREVG of an inverse transform that follows it in the same CTA.
template <int LOGM>
constexpr int last_forward_group() {
    return FftShape<LOGM>::NP >= 2 ? xgroup<LOGM>(FftShape<LOGM>::NP - 2) : 0;
}

// Two segments as the real and imaginary parts of z: point n = t + T*j is
// sample s0 + n of row x0 (re) and s1 + n of row x1 (im), zero outside
// [0, N) or when !live1.  REV: the rows hold their samples in reverse time
// (sample n at row[N - 1 - n]); the warps' reads stay contiguous.
template <int LOGM, bool REV = false>
__device__ __forceinline__ void load_pair(float2 (&v)[FftShape<LOGM>::PT], const float* x0, const float* x1,
                                          bool live1, int64_t s0, int64_t s1, int64_t N, int t) {
    using F = FftShape<LOGM>;
    if (live1 && s0 >= 0 && s1 >= 0 && s0 + F::M <= N && s1 + F::M <= N) {
        if constexpr (!REV) {
            const float* p0 = x0 + s0 + t;
            const float* p1 = x1 + s1 + t;
#pragma unroll
            for (int j = 0; j < F::PT; ++j) v[j] = make_float2(__ldg(p0 + F::T * j), __ldg(p1 + F::T * j));
        } else {
            const float* p0 = x0 + (N - 1 - s0) - t;
            const float* p1 = x1 + (N - 1 - s1) - t;
#pragma unroll
            for (int j = 0; j < F::PT; ++j) v[j] = make_float2(__ldg(p0 - F::T * j), __ldg(p1 - F::T * j));
        }
    } else {
#pragma unroll
        for (int j = 0; j < F::PT; ++j) {
            const int64_t n0 = s0 + t + F::T * j, n1 = s1 + t + F::T * j;
            v[j].x = (n0 >= 0 && n0 < N) ? __ldg(x0 + (REV ? N - 1 - n0 : n0)) : 0.f;
            v[j].y = (live1 && n1 >= 0 && n1 < N) ? __ldg(x1 + (REV ? N - 1 - n1 : n1)) : 0.f;
        }
    }
}

// Points n >= first of each segment are outputs n - first of its block,
// samples b0 + [0, m0) of row y0 (real parts) and b1 + [0, m1) of row y1
// (imaginary parts); REV: rows in reverse time, as for load_pair.  Register
// j of thread t is point t + T j: one row pointer per thread, a constant
// offset per register, and one unsigned compare per store.
template <int LOGM, bool REV = false>
__device__ __forceinline__ void store_pair(const float2 (&v)[FftShape<LOGM>::PT], float* y0, float* y1, int64_t b0,
                                           int64_t b1, int64_t N, int first, int m0, int m1, int t) {
    using F = FftShape<LOGM>;
    float* p0 = REV ? y0 + (N - 1 - b0 + first) - t : y0 + (b0 - first) + t;
    float* p1 = REV ? y1 + (N - 1 - b1 + first) - t : y1 + (b1 - first) + t;
    const int o0 = t - first;
#pragma unroll
    for (int j = 0; j < F::PT; ++j) {
        const int o = o0 + F::T * j;
        if ((unsigned)o < (unsigned)m0) p0[REV ? -F::T * j : F::T * j] = v[j].x;
        if ((unsigned)o < (unsigned)m1) p1[REV ? -F::T * j : F::T * j] = v[j].y;
    }
}

// store_pair (forward time) with the MSE fused: each output y also gives
// d = y - t (t the target at the same place) and the gradient gs d (rows
// t0 / t1 and g0 / g1 laid out like y0 / y1); returns this thread's sum of
// d^2 (FP32, at most 2 PT terms).  KEEP_G: v is left holding the gradient at
// every output position and zero elsewhere (the block's gradient window,
// ready for its own transform).
template <int LOGM, bool KEEP_G = false>
__device__ __forceinline__ float store_pair_mse(float2 (&v)[FftShape<LOGM>::PT], float* y0, float* y1,
                                                const float* t0, const float* t1, float* g0, float* g1, int64_t b0,
                                                int64_t b1, int first, int m0, int m1, int t, float gs) {
    using F = FftShape<LOGM>;
    const int64_t o0 = b0 - first + t, o1 = b1 - first + t;
    float* py0 = y0 + o0;
    float* py1 = y1 + o1;
    const float* pt0 = t0 + o0;
    const float* pt1 = t1 + o1;
    float* pg0 = g0 + o0;
    float* pg1 = g1 + o1;
    const int oo = t - first;
    float acc = 0.f;
    // four registers' targets in flight at a time
#pragma unroll
    for (int j0 = 0; j0 < F::PT; j0 += 4) {
        float tv0[4], tv1[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = oo + F::T * (j0 + j);
            tv0[j] = (unsigned)o < (unsigned)m0 ? __ldcs(pt0 + F::T * (j0 + j)) : 0.f;
            tv1[j] = (unsigned)o < (unsigned)m1 ? __ldcs(pt1 + F::T * (j0 + j)) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = oo + F::T * (j0 + j);
            float ga = 0.f, gb = 0.f;
            if ((unsigned)o < (unsigned)m0) {
                py0[F::T * (j0 + j)] = v[j0 + j].x;
                const float d = v[j0 + j].x - tv0[j];
                ga = d * gs;
                pg0[F::T * (j0 + j)] = ga;
                acc = fmaf(d, d, acc);
            }
            if ((unsigned)o < (unsigned)m1) {
                py1[F::T * (j0 + j)] = v[j0 + j].y;
                const float d = v[j0 + j].y - tv1[j];
                gb = d * gs;
                pg1[F::T * (j0 + j)] = gb;
                acc = fmaf(d, d, acc);
            }
            if constexpr (KEEP_G) v[j0 + j] = make_float2(ga, gb);
        }
    }
    return acc;
}

}  // namespace
}  // namespace tfx
