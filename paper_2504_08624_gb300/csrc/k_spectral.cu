// Training kernels for chains run by their composite response (the spectral
// route of a trainable plan).  The chain is one linear time-invariant filter
// with impulse response h (TorchFX Sec. 3: the pipe composes the stages), so
// for L = sum_c sum_n g[c][n] y[c][n] and every coefficient theta:
//     dL/dtheta = sum_(j >= 0) (dh/dtheta)[j] r[j],
//     r[j]      = sum_c sum_n g[c][n] x[c][n - j]     (cross-correlation of the
//                                                      upstream gradient and
//                                                      the input, lags >= 0)
// and dL/dx is the chain applied to g in reverse time.  r is accumulated in
// the frequency domain by blocks: block b of a channel pair takes the
// gradient samples [bB, bB + B) at positions [J, M) of an M-point sequence
// (zeros before) and the input window [bB - J, bB + B); the circular
// correlation of the two equals the block's share of r at lags 0..J.  With
// two channels as the real and imaginary parts of each sequence,
// Zg conj(Zx) = S + i T where S (the wanted sum over both channels) and T are
// both spectra of real sequences, so S = (P + conj(P mirrored)) / 2 once P is
// summed over every block.  The gradients are then inner products with the
// derivative spectra, taken from the sections' coefficients in closed form at
// each bin (FP64): for section s with A_s = 1 + a1 z + a2 z^2 and
// B_s = b0 + b1 z + b2 z^2 (a0-normalised, z = e^(-i w)), H = prod_s B_s/A_s
// times the FIR's spectrum F,
//     dH/db_k = z^k F prod_(j != s) H_j / A_s,   dH/da_k = -z^k H / A_s,
// and for the FIR taps dL/dh_k is the inverse transform of conj(prod_s H_s) S
// at sample k.  The derivative responses decay with the chain's poles, so
// lags beyond J (where the circular correlation is not r) meet only their
// negligible tails.
#include <algorithm>

#include "fft_core.cuh"

namespace tfx {
namespace {

constexpr double TWO_PI = 6.283185307179586476925286766559;

// Storage index i of the spectra (float4 q of thread t, halves e: i = 2(qT + t)
// + e) <-> transform position k = 16t + 2q + e (the forward transform's output
// slot), whose frequency bin is bitrev_m(k).
__device__ __forceinline__ int pos_of_storage(int i, int T) {
    const int e = i & 1, q = (i >> 1) / T, t = (i >> 1) % T;
    return 16 * t + 2 * q + e;
}
__device__ __forceinline__ int storage_of_pos(int k, int T) {
    const int t = k >> 4, q = (k & 15) >> 1, e = k & 1;
    return 2 * (q * T + t) + e;
}
__device__ __forceinline__ int bitrev_bits(int k, int m) { return (int)(__brev((unsigned)k) >> (32 - m)); }

struct dcplx {
    double re, im;
};
__device__ __forceinline__ dcplx dmul(dcplx a, dcplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
// 1 / b: the reciprocal of |b|^2 from the FP32 estimate refined by two
// Newton steps (each doubles the correct bits: 24 -> 48 -> full), cheaper
// than an FP64 division on this part; |b|^2 stays within FP32 range for the
// denominators of stable sections (>= (1 - r)^4 with r <= 0.999).
__device__ __forceinline__ dcplx drecip(dcplx b) {
    const double d = b.re * b.re + b.im * b.im;
    double r = (double)__frcp_rn((float)d);
    r = r * fma(-d, r, 2.0);
    r = r * fma(-d, r, 2.0);
    return {b.re * r, -b.im * r};
}

// Section s's numerator and denominator at z (raw row: the a0 cancels in the
// ratio; the derivative formulas take the normalised coefficients).
__device__ __forceinline__ void section_at(const double* r, dcplx z1, dcplx z2, dcplx& Bn, dcplx& An) {
    const double inv = 1.0 / r[3];
    Bn = {r[0] * inv + r[1] * inv * z1.re + r[2] * inv * z2.re, r[1] * inv * z1.im + r[2] * inv * z2.im};
    An = {1.0 + r[4] * inv * z1.re + r[5] * inv * z2.re, r[4] * inv * z1.im + r[5] * inv * z2.im};
}

// Block correlation spectra, accumulated per CTA over its (channel pair,
// block) items and written as one M-point partial in storage layout.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16, LOGM <= 12 ? 2 : 1) k_chain_xcorr(XcorrArgs a) {
    using F = FftShape<LOGM>;
    static_assert(F::PT == 16, "the spectral kernels use 4096- and 8192-point transforms");
    extern __shared__ float2 sb[];
    float2* zx = sb + (F::M + F::M / 16);  // the input window's spectrum, each thread its own slots
    const int t = threadIdx.x;
    float2 acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = make_float2(0.f, 0.f);
    const unsigned nbpc = (unsigned)a.nbpc;
    for (unsigned it = blockIdx.x; it < (unsigned)a.items; it += gridDim.x) {
        const unsigned r = it / nbpc, b = it - r * nbpc;
        const int64_t c0 = 2 * (int64_t)r;
        const bool live1 = c0 + 1 < a.C;
        const int64_t n0 = (int64_t)b * a.B;
        float2 v[16];
        __syncthreads();  // the previous transform's exchanges are done with sb
        load_pair<LOGM>(v, a.x + c0 * a.ldx, a.x + (live1 ? c0 + 1 : c0) * a.ldx, live1, n0 - a.J, n0 - a.J, a.N, t);
        forward_from<LOGM, 0>(v, a.tw, sb, t);
#pragma unroll
        for (int j = 0; j < 16; ++j) zx[j * F::T + t] = v[j];
        // gradient samples n0 + (p - J) at positions p >= J, zeros before
        // (lim of them in this block)
        const int lim = (int)(a.N - n0 < a.B ? a.N - n0 : a.B);
        const float* g0 = a.g + c0 * a.ldg + (n0 - a.J) + t;
        const float* g1 = live1 ? g0 + a.ldg : g0;
        const int o0 = t - a.J;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const bool in = (unsigned)(o0 + F::T * j) < (unsigned)lim;
            v[j] = make_float2(in ? __ldg(g0 + F::T * j) : 0.f, (in && live1) ? __ldg(g1 + F::T * j) : 0.f);
        }
        __syncthreads();
        forward_from<LOGM, 0>(v, a.tw, sb, t);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float2 w = zx[j * F::T + t];
            acc[j].x = fmaf(v[j].x, w.x, fmaf(v[j].y, w.y, acc[j].x));
            acc[j].y = fmaf(v[j].y, w.x, fmaf(-v[j].x, w.y, acc[j].y));
        }
    }
    float4* out = reinterpret_cast<float4*>(a.part + (int64_t)blockIdx.x * F::M) + t;
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q * F::T] = make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y);
}

// P = sum of the CTAs' partials, in FP64 (storage layout).  Block b takes
// bins [32b, 32b + 32): warp w sums partials w, w + 32, ... for its lane's
// bin (coalesced rows), then the warp sums are added in warp order.
constexpr int REDUCE_WARPS = 32;
__global__ void __launch_bounds__(32 * REDUCE_WARPS) k_xcorr_reduce(const float2* __restrict__ part, int G, int M,
                                                                   double2* __restrict__ P) {
    __shared__ double2 red[REDUCE_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    // compensated (Kahan) FP32 sums per thread: FP64 adds are scarce on this part
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    if (i < M) {
#pragma unroll 4
        for (int g = w; g < G; g += REDUCE_WARPS) {
            const float2 v = __ldcs(part + (int64_t)g * M + i);
            const float yr = v.x - cr, tr = sr + yr;
            cr = (tr - sr) - yr;
            sr = tr;
            const float yi = v.y - ci, ti = si + yi;
            ci = (ti - si) - yi;
            si = ti;
        }
    }
    red[w][lane] = make_double2((double)sr - (double)cr, (double)si - (double)ci);
    __syncthreads();
    if (w == 0 && i < M) {
        double2 s = red[0][lane];
        for (int k = 1; k < REDUCE_WARPS; ++k) s.x += red[k][lane].x, s.y += red[k][lane].y;
        P[i] = s;
    }
}

// Complex shuffles (each part a 64-bit shuffle).
__device__ __forceinline__ dcplx shfl_up_c(dcplx v, int d) {
    return {__shfl_up_sync(0xffffffffu, v.re, d), __shfl_up_sync(0xffffffffu, v.im, d)};
}
__device__ __forceinline__ dcplx shfl_down_c(dcplx v, int d) {
    return {__shfl_down_sync(0xffffffffu, v.re, d), __shfl_down_sync(0xffffffffu, v.im, d)};
}
__device__ __forceinline__ dcplx shfl_c(dcplx v, int src) {
    return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

__device__ __forceinline__ float2 fshfl_up(float2 v, int d) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 fshfl_down(float2 v, int d) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 fshfl(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float2 frecip(float2 b) {
    const float d = 1.0f / fmaf(b.x, b.x, b.y * b.y);
    return make_float2(b.x * d, -b.y * d);
}

// A section's numerator B(z) and denominator A(z) (a0-normalised
// coefficients) at z = zt[bin]: evaluated in FP64, where the cancellation
// near a pole or a zero happens, then rounded to FP32 (relative error
// ~6e-8 however small |A| is); the products and quotients that follow are
// well conditioned and run in FP32 (FP64 throughput is scarce on this part;
// measured on CPU against all-FP64: <= 1e-6 of each stage's largest
// gradient on the test chains).
__device__ __forceinline__ void section_poly(const double2* __restrict__ zt, int bin, double b0, double b1,
                                             double b2, double a1, double a2, float2& Bn, float2& An) {
    const double2 z = zt[bin];
    const double z2r = z.x * z.x - z.y * z.y, z2i = 2.0 * z.x * z.y;
    Bn = make_float2((float)(b0 + b1 * z.x + b2 * z2r), (float)(b1 * z.y + b2 * z2i));
    An = make_float2((float)(1.0 + a1 * z.x + a2 * z2r), (float)(a1 * z.y + a2 * z2i));
}

// Composite spectrum in the filter's layout (storage index i, 1/M folded
// in): the FIR's spectrum Hf (already scaled) times prod_s B_s / A_s at the
// bin of i, one lane per (bin, section) as in k_chain_grads_sec.
__global__ void __launch_bounds__(128) k_chain_spectrum(const double* __restrict__ raw, int S,
                                                        const float2* __restrict__ Hf, const double2* __restrict__ zt,
                                                        int m, float2* __restrict__ H) {
    const int M = 1 << m, T = M / 16;
    const int lane = threadIdx.x & 31;
    const int NB = 32 / S, slot = lane / S, sec = lane % S;
    const bool active = slot < NB;
    const double* r = raw + 6 * (active ? sec : 0);
    const double inv0 = 1.0 / r[3];
    const double b0 = r[0] * inv0, b1 = r[1] * inv0, b2 = r[2] * inv0, a1 = r[4] * inv0, a2 = r[5] * inv0;
    const int gi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int i = gi * NB + slot;
    const bool live = active && i < M;
    const int ii = live ? i : 0;
    const int bin = bitrev_bits(pos_of_storage(ii, T), m);
    float2 Bn, An;
    section_poly(zt, bin, b0, b1, b2, a1, a2, Bn, An);
    float2 pin = cmul(Bn, frecip(An));
    for (int d = 1; d < S; d <<= 1) {
        const float2 u = fshfl_up(pin, d);
        if (sec >= d) pin = cmul(u, pin);
    }
    if (live && sec == S - 1) H[i] = cmul(Hf[i], pin);
}

// Section coefficient gradients (a0-normalised b0 b1 b2 a1 a2 per section):
// the section polynomials in FP64, the products in FP32 (section_poly), the
// sums in FP64.  A warp takes NB = floor(32 / S) bins at a time with one lane per
// (bin, section): lane l is section l % S of bin slot l / S, so each lane
// evaluates one section, the products over the other sections come from
// segmented prefix and suffix scans across the bin's S lanes, and a lane
// accumulates the gradient terms of one fixed section over all the bins it
// visits (enough warps per SM to hide the latency).  Each block writes its
// sums to bpart[block][5 S] (k_spectral_finalize adds them in block order,
// so the result does not depend on the blocks' timing).  With wfir
// set, also conj(C) S at each bin (C = prod_s H_s, the cascades' spectrum)
// for the FIR tap gradients, in storage layout.
constexpr int GRADS_WARPS = 4;
__global__ void __launch_bounds__(32 * GRADS_WARPS) k_chain_grads_sec(
    const double2* __restrict__ P, const double* __restrict__ raw, int S, const float2* __restrict__ Hf,
    const double2* __restrict__ zt, int m, double* __restrict__ bpart, float2* __restrict__ wfir) {
    __shared__ double red[GRADS_WARPS][32][5];
    const int M = 1 << m, T = M / 16;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int NB = 32 / S, slot = lane / S, sec = lane % S;
    const bool active = slot < NB;
    const int first = slot * S;  // the bin's section-0 lane
    // this lane's section, a0-normalised
    const double* r = raw + 6 * (active ? sec : 0);
    const double inv0 = 1.0 / r[3];
    const double b0 = r[0] * inv0, b1 = r[1] * inv0, b2 = r[2] * inv0, a1 = r[4] * inv0, a2 = r[5] * inv0;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int groups = (M + NB - 1) / NB;
    for (int gi = blockIdx.x * GRADS_WARPS + warp; gi < groups; gi += gridDim.x * GRADS_WARPS) {
        const int i = gi * NB + slot;  // storage index of this lane's bin
        const bool live = active && i < M;
        const int ii = live ? i : 0;
        const int bin = bitrev_bits(pos_of_storage(ii, T), m);
        const int mir = (M - bin) & (M - 1);
        const double2 p = P[ii], pm = P[storage_of_pos(bitrev_bits(mir, m), T)];
        const float2 Sv = make_float2((float)(0.5 * (p.x + pm.x)), (float)(0.5 * (p.y - pm.y)));
        const double2 zb = zt[bin];
        const float2 z1 = make_float2((float)zb.x, (float)zb.y), z2 = cmul(z1, z1);
        const float2 F = make_float2(Hf[ii].x * (float)M, Hf[ii].y * (float)M);
        float2 Bn, An;
        section_poly(zt, bin, b0, b1, b2, a1, a2, Bn, An);
        const float2 iA = frecip(An);
        const float2 Hs = cmul(Bn, iA);
        // inclusive prefix and suffix products over the bin's sections
        float2 pin = Hs, sin_ = Hs;
        for (int d = 1; d < S; d <<= 1) {
            const float2 u = fshfl_up(pin, d), w = fshfl_down(sin_, d);
            if (sec >= d) pin = cmul(u, pin);
            if (sec + d < S) sin_ = cmul(sin_, w);
        }
        float2 pre = fshfl_up(pin, 1), suf = fshfl_down(sin_, 1);
        if (sec == 0) pre = make_float2(1.f, 0.f);
        if (sec == S - 1) suf = make_float2(1.f, 0.f);
        const float2 Cs = fshfl(pin, first + S - 1);  // the product over every section
        if (!live) continue;
        if (wfir && sec == 0) wfir[i] = cmul(make_float2(Cs.x, -Cs.y), Sv);
        const float2 q0 = cmul(cmul(F, cmul(pre, suf)), iA);  // dH/db_0 = F prod_(j != s) H_j / A_s
        const float2 q1 = cmul(q0, z1), q2 = cmul(q0, z2);
        const float2 h0 = cmul(cmul(F, Cs), iA);              // -dH/da_k = z^k H / A_s
        const float2 h1 = cmul(h0, z1), h2 = cmul(h0, z2);
        // Re(conj(d) S), added in FP64
        acc[0] += (double)fmaf(q0.x, Sv.x, q0.y * Sv.y);
        acc[1] += (double)fmaf(q1.x, Sv.x, q1.y * Sv.y);
        acc[2] += (double)fmaf(q2.x, Sv.x, q2.y * Sv.y);
        acc[3] -= (double)fmaf(h1.x, Sv.x, h1.y * Sv.y);
        acc[4] -= (double)fmaf(h2.x, Sv.x, h2.y * Sv.y);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) red[warp][lane][k] = acc[k];
    __syncthreads();
    // block sums per (section, term), in warp and slot order
    const double invM = 1.0 / (double)M;
    for (int q = threadIdx.x; q < 5 * S; q += blockDim.x) {
        const int sq = q / 5, k = q % 5;
        double v = 0.0;
        for (int w = 0; w < GRADS_WARPS; ++w)
            for (int b = 0; b < NB; ++b) v += red[w][b * S + sq][k];
        bpart[(int64_t)blockIdx.x * 5 * S + q] = v * invM;
    }
}

// The section gradients from the blocks' partial sums, then the a0 chain
// rule to the raw rows: block s (one per section), warp k (of 5) adds term
// k over the blocks b = lane, lane + 32, ... and then by a fixed shuffle
// tree; with G the five sums of section s (normalised b0 b1 b2 a1 a2) and r
// its raw row, dL/db_k = G_k / a0, dL/da_k = G_(k+2) / a0 (k = 1, 2) and
// dL/da0 = -(sum of the raw coefficients times their G) / a0^2.
__global__ void __launch_bounds__(160) k_spectral_finalize(const double* __restrict__ bpart, int nblk, int S,
                                                           const double* __restrict__ raw,
                                                           const int64_t* __restrict__ dst,
                                                           double* __restrict__ dcoef) {
    __shared__ double G[5];
    const int sec = blockIdx.x, k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v = 0.0;
    for (int b = lane; b < nblk; b += 32) v += __ldcg(bpart + (int64_t)b * 5 * S + 5 * sec + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) G[k] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double* r = raw + 6 * sec;
        const double inv = 1.0 / r[3];
        double* o = dcoef + dst[sec];
        o[0] = G[0] * inv;
        o[1] = G[1] * inv;
        o[2] = G[2] * inv;
        o[4] = G[3] * inv;
        o[5] = G[4] * inv;
        o[3] = -(r[0] * G[0] + r[1] * G[1] + r[2] * G[2] + r[4] * G[3] + r[5] * G[4]) * inv * inv;
    }
}

// Inverse transform of a spectrum given in storage layout (position
// 16t + j of thread t read from its storage index): afterwards register j of
// thread t holds sample t + T j.
template <int LOGM>
__device__ __forceinline__ void inverse_of_storage(const float2* __restrict__ W, float2 (&v)[16],
                                                   const float2* __restrict__ tw, float2* sb, int t) {
    using F = FftShape<LOGM>;
    static_assert(F::PT == 16, "the spectral kernels use 4096- and 8192-point transforms");
    const float4* w4 = reinterpret_cast<const float4*>(W) + t;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 w = w4[q * F::T];
        v[2 * q] = make_float2(w.x, w.y);
        v[2 * q + 1] = make_float2(w.z, w.w);
    }
    inverse_from<LOGM, F::NP - 1>(v, tw, sb, t);
}

// FIR tap gradients: dL/dh_k = (1/M) sum_bins conj(C) S e^(+i w k) (C the
// cascades' spectrum), the inverse transform of wfir at samples 0..L-1.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16, 1) k_chain_grads_fir(const float2* __restrict__ wfir,
                                                                         const float2* __restrict__ tw, int L,
                                                                         double* __restrict__ dh) {
    using F = FftShape<LOGM>;
    static_assert(F::PT == 16, "the spectral kernels use 4096- and 8192-point transforms");
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    float2 v[16];
    inverse_of_storage<LOGM>(wfir, v, tw, sb, t);
    const double invM = 1.0 / (double)F::M;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int n = t + F::T * j;
        if (n < L) dh[n] = (double)v[j].x * invM;
    }
}

// Decay check of a composite spectrum H (storage layout, 1/M folded in): its
// inverse transform is the chain's impulse response aliased M-periodically;
// the absolute sum of samples J+1 .. M-1 (which the overlap-save blocks would
// wrap onto other outputs) above 1e-4 of the whole sets TFX_ERR_DECAY.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / 16, 1) k_chain_tail(const float2* __restrict__ H,
                                                                    const float2* __restrict__ tw, int J,
                                                                    int* __restrict__ status) {
    using F = FftShape<LOGM>;
    static_assert(F::PT == 16, "the spectral kernels use 4096- and 8192-point transforms");
    extern __shared__ float2 sb[];
    __shared__ float red[2][32];
    const int t = threadIdx.x;
    float2 v[16];
    inverse_of_storage<LOGM>(H, v, tw, sb, t);
    float tot = 0.f, tail = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int n = t + F::T * j;
        const float a = fabsf(v[j].x);
        tot += a;
        if (n > J) tail += a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        tail += __shfl_xor_sync(0xffffffffu, tail, o);
    }
    if ((t & 31) == 0) {
        red[0][t >> 5] = tot;
        red[1][t >> 5] = tail;
    }
    __syncthreads();
    if (t == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < F::T / 32; ++w) a += red[0][w], b += red[1][w];
        if (!(b <= 1e-4 * a)) atomicCAS(status, 0, (int)TFX_ERR_DECAY);
    }
}

template <int LOGM>
cudaError_t launch_xcorr_log(const XcorrArgs& a, int grid, cudaStream_t s) {
    constexpr int T = (1 << LOGM) / 16;
    const size_t smem = xcorr_smem_bytes(1 << LOGM);
    k_chain_xcorr<LOGM><<<(unsigned)grid, T, smem, s>>>(a);
    return cudaGetLastError();
}

template <int LOGM>
cudaError_t prepare_spectral_log() {
    const int smem = (int)fir_fft_smem_bytes(1 << LOGM);
    cudaError_t e = cudaFuncSetAttribute(k_chain_xcorr<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)xcorr_smem_bytes(1 << LOGM));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chain_grads_fir<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chain_tail<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

}  // namespace

size_t xcorr_smem_bytes(int M) { return fir_fft_smem_bytes(M) + (size_t)M * sizeof(float2); }

int xcorr_ctas_per_sm(int m) { return m <= 12 ? 2 : 1; }

cudaError_t prepare_spectral(int m) {
    switch (m) {
        case 12: return prepare_spectral_log<12>();
        case 13: return prepare_spectral_log<13>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_chain_xcorr(int m, const XcorrArgs& a, int grid, cudaStream_t s) {
    if (a.items > INT32_MAX) return cudaErrorInvalidValue;  // 32-bit item indices
    switch (m) {
        case 12: return launch_xcorr_log<12>(a, grid, s);
        case 13: return launch_xcorr_log<13>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_xcorr_reduce(const float2* part, int G, int M, double2* P, cudaStream_t s) {
    k_xcorr_reduce<<<(unsigned)((M + 31) / 32), 32 * REDUCE_WARPS, 0, s>>>(part, G, M, P);
    return cudaGetLastError();
}

cudaError_t launch_chain_spectrum(const double* raw, int S, const float2* Hf, const double2* zt, int m, float2* H,
                                  cudaStream_t s) {
    const int M = 1 << m;
    if (S < 1 || S > SPEC_SMAX) return cudaErrorInvalidValue;
    const int warps = (M + 32 / S - 1) / (32 / S);
    k_chain_spectrum<<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(raw, S, Hf, zt, m, H);
    return cudaGetLastError();
}

cudaError_t launch_chain_tail(int m, const float2* H, const float2* tw, int J, int* status, cudaStream_t s) {
    const size_t smem = fir_fft_smem_bytes(1 << m);
    switch (m) {
        case 12: k_chain_tail<12><<<1, 256, smem, s>>>(H, tw, J, status); break;
        case 13: k_chain_tail<13><<<1, 512, smem, s>>>(H, tw, J, status); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Blocks of the section-gradient kernel: about 6 warps per SM of bin
// groups, at most one group per warp.
int chain_grads_blocks(int m, int S) {
    const int groups = ((1 << m) + 32 / S - 1) / (32 / S);
    return std::max(1, std::min((groups + GRADS_WARPS - 1) / GRADS_WARPS, 2 * 152));
}

size_t chain_grads_scratch_bytes(int m, int S) { return (size_t)chain_grads_blocks(m, S) * 5 * S * sizeof(double); }

cudaError_t launch_spectral_finalize(int m, const void* scratch, int S, const double* raw, const int64_t* dst,
                                     double* dcoef, cudaStream_t s) {
    if (S < 1 || S > SPEC_SMAX) return cudaErrorInvalidValue;
    k_spectral_finalize<<<(unsigned)S, 160, 0, s>>>(static_cast<const double*>(scratch), chain_grads_blocks(m, S), S,
                                                    raw, dst, dcoef);
    return cudaGetLastError();
}

cudaError_t launch_chain_grads(int m, const double2* P, const double* raw, int S, const float2* Hf,
                               const double2* zt, const float2* tw, int L, void* scratch, float2* wfir, double* dh,
                               cudaStream_t s) {
    if (S < 1 || S > SPEC_SMAX) return cudaErrorInvalidValue;
    const int M = 1 << m;
    double* bpart = static_cast<double*>(scratch);
    k_chain_grads_sec<<<(unsigned)chain_grads_blocks(m, S), 32 * GRADS_WARPS, 0, s>>>(P, raw, S, Hf, zt, m, bpart,
                                                                                   dh ? wfir : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !dh) return e;
    const size_t smem = fir_fft_smem_bytes(M);
    switch (m) {
        case 12: k_chain_grads_fir<12><<<1, 256, smem, s>>>(wfir, tw, L, dh); break;
        case 13: k_chain_grads_fir<13><<<1, 512, smem, s>>>(wfir, tw, L, dh); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace tfx
