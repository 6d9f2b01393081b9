// FIR by FFT overlap-save (the FFT route for long FIRs): y[n] = sum_k h[k] x[n-k].
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
// spectrum of h is stored in that order with the 1/M scale folded in, so the
// product needs no permutation, and the inverse runs the passes backwards
// (conjugate twiddles, then the DIT G-point DFT), ending in natural order in
// the layout the input was loaded in: point t + T*j in register j, so both the
// input loads and the output stores are coalesced.  A group's twiddle
// w^k is applied as the product of w^(2^b) over the set bits b of k, each
// read from a table of e^(-2 pi i k / M), k < M/2, computed in FP64 at plan
// time (at most four roundings per point and pass).
#include "tfx_common.cuh"

namespace tfx {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
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
// v[OFF + q*ST], q < G; butterflies q = Q, Q+1, ... by recursion.
template <int G, int ST, int OFF, int H, bool INV, int Q = 0>
__device__ __forceinline__ void stage(float2 (&v)[16]) {
    if constexpr (Q < G) {
        if constexpr ((Q / H) % 2 == 0) {
            constexpr int i0 = OFF + Q * ST, i1 = OFF + (Q + H) * ST;
            const float2 a = v[i0];
            if constexpr (!INV) {  // DIF: (a, c) -> (a + c, (a - c) w)
                const float2 c = v[i1];
                v[i0] = cadd(a, c);
                v[i1] = twc<Q % H, 2 * H, false>(csub(a, c));
            } else {  // DIT: (a, c) -> (a + c w*, a - c w*)
                const float2 c = twc<Q % H, 2 * H, true>(v[i1]);
                v[i0] = cadd(a, c);
                v[i1] = csub(a, c);
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

__host__ __device__ constexpr int brev(int q, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((q >> b) & 1) << (bits - 1 - b);
    return r;
}

// Multiply every slot q of the group v[OFF + q*ST] whose exponent bitrev(q)
// has bit B set by w (INV: by conj(w)).
template <int G, int ST, int OFF, int B, bool INV, int Q = 1>
__device__ __forceinline__ void apply_bit(float2 (&v)[16], float2 w) {
    if constexpr (Q < G) {
        constexpr int RB = G == 16 ? 4 : G == 8 ? 3 : G == 4 ? 2 : 1;
        constexpr int k = brev(Q, RB), i = OFF + Q * ST;
        if constexpr ((k >> B) & 1) v[i] = INV ? cmulc(v[i], w) : cmul(v[i], w);
        apply_bit<G, ST, OFF, B, INV, Q + 1>(v, w);
    }
}

// Multiply slot q of the group v[OFF + q*ST] by w^bitrev(q) (INV: its
// conjugate) in factored form: w^k = prod over the set bits b of k of
// w^(2^b) = tw[2^b * e]; no table of all powers is held in registers.
template <int G, int ST, int OFF, bool INV>
__device__ __forceinline__ void twiddle_group(float2 (&v)[16], const float2* __restrict__ tw, int e) {
    if constexpr (G >= 16) apply_bit<G, ST, OFF, 3, INV>(v, __ldg(tw + 8 * e));
    if constexpr (G >= 8) apply_bit<G, ST, OFF, 2, INV>(v, __ldg(tw + 4 * e));
    if constexpr (G >= 4) apply_bit<G, ST, OFF, 1, INV>(v, __ldg(tw + 2 * e));
    apply_bit<G, ST, OFF, 0, INV>(v, __ldg(tw + e));
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
};

// Position of register j of thread t in pass P.  Pass 0 (span M): point
// t + T*j.  A radix-16 pass over span S (sub = S/16): point
// (t / sub) * S + t % sub + j * sub.
template <int LOGM, int P>
__device__ __forceinline__ int ppos(int t, int j) {
    using F = FftShape<LOGM>;
    if constexpr (P == 0) {
        return t + F::T * j;
    } else {
        constexpr int S = F::span(P), sub = S / 16;
        return (t / sub) * S + (t % sub) + j * sub;
    }
}

// First pass when G0 < 16: groups c < 16/G0, slot q of group c in register
// c + q*(16/G0), group position i = t + T*c.
template <int LOGM, bool INV, int C = 0>
__device__ __forceinline__ void first_groups(float2 (&v)[16], const float2* __restrict__ tw, int t) {
    using F = FftShape<LOGM>;
    constexpr int G = F::G0, NG = 16 / G;
    if constexpr (C < NG) {
        const int e = t + F::T * C;  // i * (M / S) with S = M
        if constexpr (!INV) {
            dft_dif<G, NG, C>(v);
            twiddle_group<G, NG, C, false>(v, tw, e);
        } else {
            twiddle_group<G, NG, C, true>(v, tw, e);
            dft_dit<G, NG, C>(v);
        }
        first_groups<LOGM, INV, C + 1>(v, tw, t);
    }
}

template <int LOGM, int P, bool INV>
__device__ __forceinline__ void run_pass(float2 (&v)[16], const float2* __restrict__ tw, int t) {
    using F = FftShape<LOGM>;
    if constexpr (P == 0 && F::R0 != 0) {
        first_groups<LOGM, INV>(v, tw, t);
    } else {
        constexpr int S = F::span(P), sub = S / 16;
        const int e = (t % sub) * (F::M / S);
        if constexpr (!INV) {
            dft_dif<16, 1, 0>(v);
            if constexpr (sub > 1) twiddle_group<16, 1, 0, false>(v, tw, e);
        } else {
            if constexpr (sub > 1) twiddle_group<16, 1, 0, true>(v, tw, e);
            dft_dit<16, 1, 0>(v);
        }
    }
}

// Move the points from pass P's layout to pass Q's through shared memory.
template <int LOGM, int P, int Q>
__device__ __forceinline__ void exchange(float2 (&v)[16], float2* sb, int t) {
#pragma unroll
    for (int j = 0; j < 16; ++j) sb[pad(ppos<LOGM, P>(t, j))] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = sb[pad(ppos<LOGM, Q>(t, j))];
    __syncthreads();
}

template <int LOGM, int P>
__device__ __forceinline__ void forward_from(float2 (&v)[16], const float2* __restrict__ tw, float2* sb, int t) {
    run_pass<LOGM, P, false>(v, tw, t);
    if constexpr (P + 1 < FftShape<LOGM>::NP) {
        exchange<LOGM, P, P + 1>(v, sb, t);
        forward_from<LOGM, P + 1>(v, tw, sb, t);
    }
}

template <int LOGM, int P>
__device__ __forceinline__ void inverse_from(float2 (&v)[16], const float2* __restrict__ tw, float2* sb, int t) {
    run_pass<LOGM, P, true>(v, tw, t);
    if constexpr (P > 0) {
        exchange<LOGM, P, P - 1>(v, sb, t);
        inverse_from<LOGM, P - 1>(v, tw, sb, t);
    }
}

template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16) k_fir_fft(FirFftArgs a) {
    using F = FftShape<LOGM>;
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    const int64_t k0 = 2 * (int64_t)blockIdx.x;
    const bool live1 = k0 + 1 < a.nb;
    const int64_t c0 = k0 / a.nbpc, c1 = live1 ? (k0 + 1) / a.nbpc : c0;
    const int64_t n00 = (k0 % a.nbpc) * (int64_t)a.B, n01 = live1 ? ((k0 + 1) % a.nbpc) * (int64_t)a.B : 0;
    const int Hh = a.L - 1;
    const float* x0 = a.x + c0 * a.ldx;
    const float* x1 = a.x + c1 * a.ldx;
    float2 v[16];
    // point n = t + T*j is sample n0 - (L - 1) + n: re = block k0, im = block k0 + 1
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int n = t + F::T * j;
        const int64_t s0 = n00 - Hh + n, s1 = n01 - Hh + n;
        v[j].x = (s0 >= 0 && s0 < a.N) ? __ldg(x0 + s0) : 0.f;
        v[j].y = (live1 && s1 >= 0 && s1 < a.N) ? __ldg(x1 + s1) : 0.f;
    }
    forward_from<LOGM, 0>(v, a.tw, sb, t);
    // spectrum product: thread t holds positions 16t .. 16t + 15
    const float4* h4 = reinterpret_cast<const float4*>(a.H) + 8 * t;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 h = __ldg(h4 + q);
        v[2 * q] = cmul(v[2 * q], make_float2(h.x, h.y));
        v[2 * q + 1] = cmul(v[2 * q + 1], make_float2(h.z, h.w));
    }
    inverse_from<LOGM, F::NP - 1>(v, a.tw, sb, t);
    // the last B points of each segment are the block's outputs
    const int64_t m0 = a.N - n00 < a.B ? a.N - n00 : a.B;
    const int64_t m1 = live1 ? (a.N - n01 < a.B ? a.N - n01 : a.B) : 0;
    float* y0 = a.y + c0 * a.ldy + n00;
    float* y1 = a.y + c1 * a.ldy + n01;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int o = t + F::T * j - Hh;  // output index within the block
        if (o >= 0) {
            if (o < m0) y0[o] = v[j].x;
            if (o < m1) y1[o] = v[j].y;
        }
    }
}

template <int LOGM>
cudaError_t launch_log(const FirFftArgs& a, cudaStream_t s) {
    const int64_t ctas = (a.nb + 1) / 2;
    k_fir_fft<LOGM><<<(unsigned)ctas, (1 << LOGM) / 16, fir_fft_smem_bytes(1 << LOGM), s>>>(a);
    return cudaGetLastError();
}

template <int LOGM>
cudaError_t prepare_log() {
    return cudaFuncSetAttribute(k_fir_fft<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fir_fft_smem_bytes(1 << LOGM));
}

}  // namespace

size_t fir_fft_smem_bytes(int M) { return (size_t)(M + M / 16) * sizeof(float2); }

cudaError_t prepare_fir_fft(int M) {
    switch (M) {
        case 1024: return prepare_log<10>();
        case 2048: return prepare_log<11>();
        case 4096: return prepare_log<12>();
        case 8192: return prepare_log<13>();
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
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tfx
