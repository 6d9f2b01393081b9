// FIR by FFT overlap-save (the FFT route for long FIRs): y[n] = sum_k h[k] x[n-k].
//
// Two schemes share the transforms.  Single-block (L - 1 < 3M/4), below:
// each block's segment is transformed, multiplied by the spectrum of h and
// transformed back.  Partitioned (any L): h is cut into P partitions of
// B = M/2 taps, every input segment is transformed once (k_fir_fft_spec) and
// block b's spectrum is the sum over p of H_p Z_(b-p) (k_fir_fft_conv), with
// the two channels of a pair as the real and imaginary parts.
//
// Blocks of B = M - (L - 1) outputs; block b reads the input segment
// x[n0 - (L - 1), n0 + B) (zero outside the signal), whose circular
// convolution with h (zero-padded to M) equals the linear one in its last B
// positions.  One CTA transforms TWO blocks at once: their segments are the
// real and imaginary parts of one complex sequence z; because h is real,
// H . FFT(z) = FFT(h * x1) + i FFT(h * x2), so one complex FFT, one pointwise
// product and one inverse FFT give both blocks' outputs (real part, imaginary
// part).
//
// Register-resident radix-16 FFT.  M = 2^m (m = 10..13) points, T = M/16
// threads, 16 points per thread.  The forward transform is decimation in
// frequency in passes over spans M, M/G1, ..., 16: a first pass of radix
// G1 = 2^(m mod 4) (radix 16 when m is a multiple of 4), then radix-16
// passes.  A pass over span S = G * sub takes, for each i < sub, the G points
// i + j*sub of each span, forms their G-point DFT in registers (radix-2 DIF
// stages with constant twiddles; slot j then holds output bitrev(j)) and
// multiplies slot j by w_S^(i * bitrev(j)), w_S = e^(-2 pi i / S).  Points move
// between passes through shared memory padded by one word per 16 (no bank
// conflicts for any pass's pattern).  After the last pass (span 16) thread t
// holds points 16t..16t+15 of the spectrum in bit-reversed order; the
// spectrum of h is stored in that order with the 1/M scale folded in (float4
// q of thread t, points 16t + 2q and 16t + 2q + 1, at index q*T + t, so that
// a warp's reads are contiguous), the product needs no permutation, and the
// inverse runs the passes backwards
// (conjugate twiddles, then the DIT G-point DFT), ending in natural order in
// the layout the input was loaded in: point t + T*j in register j, so both the
// input loads and the output stores are coalesced.  Each pass with twiddles
// reads them from its own table (two slots' twiddles per 16-byte word, by
// group position), computed in FP64 at plan time and rounded once:
// consecutive threads read consecutive words, and every point takes one
// complex multiply per pass.  Complex sums and differences are packed
// two-lane FP32 instructions (real and imaginary part in one register pair).
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

// v * e^(-2 pi i P / N) (INV: e^(+2 pi i P / N)) for the constant twiddles of
// the in-register DFT (N <= 16, P < N/2): exact for P = 0 and a quarter turn.
template <int P, int N, bool INV>
__device__ __forceinline__ float2 twc(float2 v) {
    constexpr int Q = (16 / N) * P;  // sixteenths of a turn, 0..7
    if constexpr (Q == 0) {
        return v;
    } else if constexpr (Q == 4) {
        return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else {
        constexpr float C1 = 0.92387953251128674f, S1 = 0.38268343236508978f, R2 = 0.70710678118654752f;
        // cos and sin of 2 pi Q / 16
        constexpr float c = Q == 1 ? C1 : Q == 2 ? R2 : Q == 3 ? S1 : Q == 5 ? -S1 : Q == 6 ? -R2 : -C1;
        constexpr float s = Q == 1 ? S1 : Q == 2 ? R2 : Q == 3 ? C1 : Q == 5 ? C1 : Q == 6 ? R2 : S1;
        return INV ? make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.y, c, v.x * s))
                   : make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -v.x * s));
    }
}

// One radix-2 stage (half-distance H) of the G-point DFT over registers
// v[OFF + q*ST], q < G; butterflies q = Q, Q+1, ... by recursion.  Sums and
// differences are packed two-lane instructions; a quarter-turn twiddle
// (multiplication by -i or +i, which swaps the lanes) is folded into scalar
// sums and differences instead.
template <int G, int ST, int OFF, int H, bool INV, int Q = 0>
__device__ __forceinline__ void stage(float2 (&v)[16]) {
    if constexpr (Q < G) {
        if constexpr ((Q / H) % 2 == 0) {
            constexpr int i0 = OFF + Q * ST, i1 = OFF + (Q + H) * ST;
            constexpr int T16 = (16 / (2 * H)) * (Q % H);  // twiddle in sixteenths of a turn
            const float2 a = v[i0];
            const float2 c = v[i1];
            if constexpr (T16 == 0) {
                v[i0] = cadd(a, c);
                v[i1] = csub(a, c);
            } else if constexpr (T16 == 4) {
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

// G-point DFT.  DIF: natural order in, slot q holds output bitrev(q).  DIT
// (inverse, unnormalised): bit-reversed in, natural out.
template <int G, int ST, int OFF>
__device__ __forceinline__ void dft_dif(float2 (&v)[16]) {
    if constexpr (G >= 16) stage<G, ST, OFF, 8, false>(v);
    if constexpr (G >= 8) stage<G, ST, OFF, 4, false>(v);
    if constexpr (G >= 4) stage<G, ST, OFF, 2, false>(v);
    if constexpr (G >= 2) stage<G, ST, OFF, 1, false>(v);
}

template <int G, int ST, int OFF>
__device__ __forceinline__ void dft_dit(float2 (&v)[16]) {
    if constexpr (G >= 2) stage<G, ST, OFF, 1, true>(v);
    if constexpr (G >= 4) stage<G, ST, OFF, 2, true>(v);
    if constexpr (G >= 8) stage<G, ST, OFF, 4, true>(v);
    if constexpr (G >= 16) stage<G, ST, OFF, 8, true>(v);
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
template <int G, int ST, int OFF, bool INV, int Q = 1>
__device__ __forceinline__ void twiddle_group(float2 (&v)[16], const float2* __restrict__ tp, int i, int sub) {
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

template <int LOGM>
struct FftShape {
    static constexpr int M = 1 << LOGM;
    static constexpr int T = M / 16;
    static constexpr int R0 = LOGM % 4;  // first pass radix 2^R0 (0: radix 16)
    static constexpr int G0 = R0 ? 1 << R0 : 16;
    static constexpr int NP = R0 ? 1 + LOGM / 4 : LOGM / 4;  // passes
    static constexpr int span(int p) { return p == 0 ? M : (M / G0) >> (4 * (p - 1)); }
    static constexpr int radix(int p) { return p == 0 ? G0 : 16; }
    static constexpr int sub(int p) { return span(p) / radix(p); }
    // offset of pass p's twiddle table ((radix - 1) rows of `sub` entries;
    // passes with sub = 1 have none)
    static constexpr int tw_off(int p) {
        int o = 0;
        for (int q = 0; q < p; ++q)
            if (sub(q) > 1) o += (radix(q) - 1) * sub(q);
        return o;
    }
};

// Padded shared-memory position of register j of thread t in pass P, as
// base(t) + j * STRIDE.  Pass 0 (span M): point t + T*j.  A radix-16 pass over
// span S (sub = S/16, which is 256, 16 or 1): point (t / sub) * S + t % sub +
// j * sub; with sub a multiple of 16 the padding adds j * sub/16, and with
// sub = 1 the point is 16t + j, padded 17t + j.
template <int LOGM, int P>
struct Layout {
    using F = FftShape<LOGM>;
    static constexpr int S = F::span(P), SUB = P == 0 ? F::T : S / 16;
    static_assert(SUB == 1 || SUB % 16 == 0, "pass layout");
    static constexpr int STRIDE = SUB == 1 ? 1 : SUB + SUB / 16;
    __device__ static __forceinline__ int base(int t) {
        if constexpr (P == 0) {
            return pad(t);
        } else if constexpr (SUB == 1) {
            return 17 * t;
        } else {
            return pad((t / SUB) * S + t % SUB);
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
__device__ __forceinline__ void run_pass(float2 (&v)[16], const float2* __restrict__ tw, int t) {
    using F = FftShape<LOGM>;
    if constexpr (P == 0 && F::R0 != 0) {
        first_groups<LOGM, INV>(v, tw + F::tw_off(0), t);
    } else {
        constexpr int sub = F::sub(P);
        const float2* tp = tw + F::tw_off(P);
        const int i = t % sub;
        if constexpr (!INV) {
            dft_dif<16, 1, 0>(v);
            if constexpr (sub > 1) twiddle_group<16, 1, 0, false>(v, tp, i, sub);
        } else {
            if constexpr (sub > 1) twiddle_group<16, 1, 0, true>(v, tp, i, sub);
            dft_dit<16, 1, 0>(v);
        }
    }
}

// Threads that exchange points between pass p and pass p + 1 (either way):
// those of one span block of pass p, a contiguous run of span(p) / 16
// threads (all of them after the first pass).
template <int LOGM>
constexpr int xgroup(int p) {
    return p == 0 ? FftShape<LOGM>::T : FftShape<LOGM>::span(p) / 16;
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
__device__ __forceinline__ void exchange(float2 (&v)[16], float2* sb, int t) {
    constexpr int G = xgroup<LOGM>(P < Q ? P : Q);
    constexpr int PRE = PREVG > G ? PREVG : G;
    if constexpr (PREVG > 0) group_sync<LOGM, PRE>(t);
    float2* w = sb + Layout<LOGM, P>::base(t);
#pragma unroll
    for (int j = 0; j < 16; ++j) w[j * Layout<LOGM, P>::STRIDE] = v[j];
    group_sync<LOGM, G>(t);
    const float2* r = sb + Layout<LOGM, Q>::base(t);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = r[j * Layout<LOGM, Q>::STRIDE];
}

// Forward passes P.. and inverse passes ..0; PREVG is the group of the
// exchange before (0: none).  Returns nothing; the exchange group sizes are
// compile-time, so the barriers cost only what the data movement requires.
template <int LOGM, int P, int PREVG = 0>
__device__ __forceinline__ void forward_from(float2 (&v)[16], const float2* __restrict__ tw, float2* sb, int t) {
    run_pass<LOGM, P, false>(v, tw, t);
    if constexpr (P + 1 < FftShape<LOGM>::NP) {
        exchange<LOGM, P, P + 1, PREVG>(v, sb, t);
        forward_from<LOGM, P + 1, xgroup<LOGM>(P)>(v, tw, sb, t);
    }
}

template <int LOGM, int P, int PREVG = 0>
__device__ __forceinline__ void inverse_from(float2 (&v)[16], const float2* __restrict__ tw, float2* sb, int t) {
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
// x0[s0 + n] (re) and x1[s1 + n] (im), zero outside [0, N) or when !live1.
template <int LOGM>
__device__ __forceinline__ void load_pair(float2 (&v)[16], const float* x0, const float* x1, bool live1, int64_t s0,
                                          int64_t s1, int64_t N, int t) {
    using F = FftShape<LOGM>;
    if (live1 && s0 >= 0 && s1 >= 0 && s0 + F::M <= N && s1 + F::M <= N) {
        const float* p0 = x0 + s0 + t;
        const float* p1 = x1 + s1 + t;
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = make_float2(__ldg(p0 + F::T * j), __ldg(p1 + F::T * j));
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int64_t n0 = s0 + t + F::T * j, n1 = s1 + t + F::T * j;
            v[j].x = (n0 >= 0 && n0 < N) ? __ldg(x0 + n0) : 0.f;
            v[j].y = (live1 && n1 >= 0 && n1 < N) ? __ldg(x1 + n1) : 0.f;
        }
    }
}

// Points n >= first of each segment are outputs n - first of its block: the
// real parts to y0[0, m0), the imaginary parts to y1[0, m1).
template <int LOGM>
__device__ __forceinline__ void store_pair(const float2 (&v)[16], float* y0, float* y1, int first, int64_t m0,
                                           int64_t m1, int t) {
    using F = FftShape<LOGM>;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int o = t + F::T * j - first;
        if (o >= 0) {
            if (o < m0) y0[o] = v[j].x;
            if (o < m1) y1[o] = v[j].y;
        }
    }
}

// One block pair of the single-block scheme: blocks 2pr and 2pr + 1.
template <int LOGM>
__device__ __forceinline__ void fft_block_pair(const FirFftArgs& a, int64_t pr, float2* sb, int t) {
    using F = FftShape<LOGM>;
    const int Hh = a.L - 1;
    const int64_t k0 = 2 * pr;
    const bool live1 = k0 + 1 < a.nb;
    const int64_t c0 = k0 / a.nbpc, c1 = live1 ? (k0 + 1) / a.nbpc : c0;
    const int64_t n00 = (k0 % a.nbpc) * (int64_t)a.B, n01 = live1 ? ((k0 + 1) % a.nbpc) * (int64_t)a.B : 0;
    float2 v[16];
    load_pair<LOGM>(v, a.x + c0 * a.ldx, a.x + c1 * a.ldx, live1, n00 - Hh, n01 - Hh, a.N, t);
    forward_from<LOGM, 0>(v, a.tw, sb, t);
    // spectrum product: thread t holds positions 16t .. 16t + 15, stored as
    // float4 q (positions 16t + 2q, 16t + 2q + 1) at index q*T + t
    const float4* h4 = reinterpret_cast<const float4*>(a.H) + t;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 h = ld_tw4(h4 + q * F::T);
        v[2 * q] = cmul(v[2 * q], make_float2(h.x, h.y));
        v[2 * q + 1] = cmul(v[2 * q + 1], make_float2(h.z, h.w));
    }
    inverse_from<LOGM, F::NP - 1, last_forward_group<LOGM>()>(v, a.tw, sb, t);
    const int64_t m0 = a.N - n00 < a.B ? a.N - n00 : a.B;
    const int64_t m1 = live1 ? (a.N - n01 < a.B ? a.N - n01 : a.B) : 0;
    store_pair<LOGM>(v, a.y + c0 * a.ldy + n00, a.y + c1 * a.ldy + n01, Hh, m0, m1, t);
}

// Single-block overlap-save: CTA k transforms blocks 2k and 2k + 1.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16, 16384 >> LOGM) k_fir_fft(FirFftArgs a) {
    extern __shared__ float2 sb[];
    fft_block_pair<LOGM>(a, blockIdx.x, sb, threadIdx.x);
}

// Single-block overlap-save over many clips in one launch (a batch of
// composed chains sharing one transform size): CTA k maps to its clip by a
// binary search over the clips' block-pair prefix sums, then transforms that
// clip's block pair k - prefix[clip] with the clip's own spectrum.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16, 16384 >> LOGM)
    k_fir_fft_batched(const BatchFft* __restrict__ units, const int64_t* __restrict__ prefix, int nunits,
                      BatchBases bases, const float2* __restrict__ tw) {
    extern __shared__ float2 sb[];
    __shared__ int s_unit;
    const int t = threadIdx.x;
    const int64_t k = blockIdx.x;
    if (t == 0) {
        int lo = 0, hi = nunits - 1;  // the last unit whose first pair is <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (prefix[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        s_unit = lo;
    }
    __syncthreads();
    const int u = s_unit;
    const BatchFft d = units[u];
    FirFftArgs a{};
    a.x = bases.ptr(d.x_sel) + d.x_off;
    a.y = bases.ptr(d.y_sel) + d.y_off;
    a.ldx = d.N;
    a.ldy = d.N;
    a.C = d.C;
    a.N = d.N;
    a.L = d.L;
    a.M = 1 << LOGM;
    a.m = LOGM;
    a.B = d.B;
    a.nbpc = d.nbpc;
    a.nb = d.nb;
    a.H = d.H;
    a.tw = tw;
    a.P = 0;
    fft_block_pair<LOGM>(a, k - prefix[u], sb, t);
}

// Partitioned overlap-save, step 1: the spectrum of segment b of a channel
// pair, x[(b - 1) B, (b + 1) B) of channels 2r (re) and 2r + 1 (im), stored
// like H: float4 q of thread t (positions 16t + 2q, 16t + 2q + 1) at q*T + t.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16, 16384 >> LOGM) k_fir_fft_spec(FirFftArgs a) {
    using F = FftShape<LOGM>;
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    const int64_t pb = blockIdx.x, r = pb / a.nbpc, b = pb % a.nbpc;
    const int64_t c0 = 2 * r;
    const bool live1 = c0 + 1 < a.C;
    const float* x0 = a.x + c0 * a.ldx;
    const int64_t s0 = (b - 1) * (int64_t)a.B;
    float2 v[16];
    load_pair<LOGM>(v, x0, live1 ? x0 + a.ldx : x0, live1, s0, s0, a.N, t);
    forward_from<LOGM, 0>(v, a.tw, sb, t);
    float4* z = reinterpret_cast<float4*>(a.Z + pb * F::M) + t;
#pragma unroll
    for (int q = 0; q < 8; ++q) z[q * F::T] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
}

// Partitioned overlap-save, step 2: block b of a channel pair is the inverse
// transform of sum over partitions p <= b of H_p Z_(b-p) (h split into P
// partitions of B taps, h_p[k] = h[pB + k]), whose last B points are outputs
// [bB, (b + 1) B).
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16, 16384 >> LOGM) k_fir_fft_conv(FirFftArgs a) {
    using F = FftShape<LOGM>;
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    const int64_t pb = blockIdx.x, r = pb / a.nbpc, b = pb % a.nbpc;
    const int64_t c0 = 2 * r;
    const bool live1 = c0 + 1 < a.C;
    float2 v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = make_float2(0.f, 0.f);
    const int np = (int)(b + 1 < a.P ? b + 1 : a.P);
    for (int p = 0; p < np; ++p) {
        const float4* h4 = reinterpret_cast<const float4*>(a.H + (int64_t)p * F::M) + t;
        const float4* z4 = reinterpret_cast<const float4*>(a.Z + (pb - p) * F::M) + t;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 h = __ldg(h4 + q * F::T), z = __ldg(z4 + q * F::T);
            v[2 * q].x = fmaf(z.x, h.x, fmaf(-z.y, h.y, v[2 * q].x));
            v[2 * q].y = fmaf(z.x, h.y, fmaf(z.y, h.x, v[2 * q].y));
            v[2 * q + 1].x = fmaf(z.z, h.z, fmaf(-z.w, h.w, v[2 * q + 1].x));
            v[2 * q + 1].y = fmaf(z.z, h.w, fmaf(z.w, h.z, v[2 * q + 1].y));
        }
    }
    inverse_from<LOGM, F::NP - 1>(v, a.tw, sb, t);
    const int64_t n0 = b * (int64_t)a.B;
    const int64_t m0 = a.N - n0 < a.B ? a.N - n0 : a.B;
    float* y0 = a.y + c0 * a.ldy + n0;
    store_pair<LOGM>(v, y0, live1 ? y0 + a.ldy : y0, F::M - a.B, m0, live1 ? m0 : 0, t);
}

// Spectrum of a FIR (or of each of its P partitions of B taps) computed on
// the device from FP64 taps, for coefficient updates without a host round
// trip: CTA p transforms h[pB, pB + len) (len = B, or L when P = 0) zero-
// padded to M points with the same forward transform the filter uses, and
// stores it as the filter reads it: scaled by 1/M, bit-reversed, float4 q of
// thread t at q*T + t.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16, 16384 >> LOGM)
    k_fir_fft_spectrum(const double* __restrict__ taps, int L, int B, int P, const float2* __restrict__ tw,
                       float2* __restrict__ H) {
    using F = FftShape<LOGM>;
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    const int part = blockIdx.x;
    const int64_t first = P > 0 ? (int64_t)part * B : 0;
    const int len = P > 0 ? B : L;
    float2 v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int n = t + F::T * j;
        const int64_t k = first + n;
        v[j] = make_float2(n < len && k < L ? (float)taps[k] : 0.f, 0.f);
    }
    forward_from<LOGM, 0>(v, tw, sb, t);
    const float inv = 1.0f / (float)F::M;
    float4* h4 = reinterpret_cast<float4*>(H + (int64_t)part * F::M) + t;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        h4[q * F::T] = make_float4(v[2 * q].x * inv, v[2 * q].y * inv, v[2 * q + 1].x * inv, v[2 * q + 1].y * inv);
}

template <int LOGM>
cudaError_t launch_spectrum_log(const double* taps, int L, int B, int P, const float2* tw, float2* H,
                                cudaStream_t s) {
    constexpr int T = (1 << LOGM) / 16;
    const size_t smem = fir_fft_smem_bytes(1 << LOGM);
    k_fir_fft_spectrum<LOGM><<<(unsigned)(P > 0 ? P : 1), T, smem, s>>>(taps, L, B, P, tw, H);
    return cudaGetLastError();
}

template <int LOGM>
cudaError_t launch_log(const FirFftArgs& a, cudaStream_t s) {
    constexpr int T = (1 << LOGM) / 16;
    const size_t smem = fir_fft_smem_bytes(1 << LOGM);
    if (a.P == 0) {
        k_fir_fft<LOGM><<<(unsigned)((a.nb + 1) / 2), T, smem, s>>>(a);
    } else {
        const int64_t ctas = (a.C + 1) / 2 * a.nbpc;
        k_fir_fft_spec<LOGM><<<(unsigned)ctas, T, smem, s>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_fir_fft_conv<LOGM><<<(unsigned)ctas, T, smem, s>>>(a);
    }
    return cudaGetLastError();
}

template <int LOGM>
cudaError_t prepare_log() {
    const int smem = (int)fir_fft_smem_bytes(1 << LOGM);
    cudaError_t e = cudaFuncSetAttribute(k_fir_fft<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft_spec<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft_conv<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft_spectrum<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft_batched<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

}  // namespace

size_t fir_fft_smem_bytes(int M) { return (size_t)(M + M / 16) * sizeof(float2); }

cudaError_t prepare_fir_fft(int M) {
    switch (M) {
        case 1024: return prepare_log<10>();
        case 2048: return prepare_log<11>();
        case 4096: return prepare_log<12>();
        case 8192: return prepare_log<13>();
        case 16384: return prepare_log<14>();
        default: return cudaErrorInvalidValue;
    }
}

template <int LOGM>
cudaError_t launch_batched_log(const BatchFft* units, const int64_t* prefix, int nunits, int64_t ctas,
                               BatchBases bases, const float2* tw, cudaStream_t s) {
    constexpr int T = (1 << LOGM) / 16;
    const size_t smem = fir_fft_smem_bytes(1 << LOGM);
    k_fir_fft_batched<LOGM><<<(unsigned)ctas, T, smem, s>>>(units, prefix, nunits, bases, tw);
    return cudaGetLastError();
}

cudaError_t launch_fir_fft_batched(int m, const BatchFft* units, const int64_t* prefix, int nunits, int64_t ctas,
                                   BatchBases bases, const float2* tw, cudaStream_t s) {
    if (ctas <= 0 || nunits <= 0) return cudaSuccess;
    switch (m) {
        case 10: return launch_batched_log<10>(units, prefix, nunits, ctas, bases, tw, s);
        case 11: return launch_batched_log<11>(units, prefix, nunits, ctas, bases, tw, s);
        case 12: return launch_batched_log<12>(units, prefix, nunits, ctas, bases, tw, s);
        case 13: return launch_batched_log<13>(units, prefix, nunits, ctas, bases, tw, s);
        case 14: return launch_batched_log<14>(units, prefix, nunits, ctas, bases, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fir_fft_spectrum(const double* taps, int L, int M, int B, int P, const float2* tw, float2* H,
                                    cudaStream_t s) {
    switch (M) {
        case 1024: return launch_spectrum_log<10>(taps, L, B, P, tw, H, s);
        case 2048: return launch_spectrum_log<11>(taps, L, B, P, tw, H, s);
        case 4096: return launch_spectrum_log<12>(taps, L, B, P, tw, H, s);
        case 8192: return launch_spectrum_log<13>(taps, L, B, P, tw, H, s);
        case 16384: return launch_spectrum_log<14>(taps, L, B, P, tw, H, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fir_fft(const FirFftArgs& a, cudaStream_t s) {
    if (a.nb <= 0) return cudaSuccess;
    switch (a.m) {
        case 10: return launch_log<10>(a, s);
        case 11: return launch_log<11>(a, s);
        case 12: return launch_log<12>(a, s);
        case 13: return launch_log<13>(a, s);
        case 14: return launch_log<14>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tfx
