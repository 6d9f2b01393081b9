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
// Register-resident radix-16 FFT.  M = 2^m (m = 10..14) points, T = M/PT
// threads, PT = 16 points per thread (32 at m = 14).  The forward transform
// is decimation in frequency in passes over spans M, M/G1, ..., 16: a first
// pass of radix G1 = 2^(m mod 4) (radix 16 when m is a multiple of 4), then
// radix-16 passes; at m = 14 passes of radix 32, 32 and 16, each thread
// taking two 16-point groups in the last.  A pass over span S = G * sub
// takes, for each i < sub, the G points i + j*sub of each span, forms their
// G-point DFT in registers (radix-2 DIF stages with constant twiddles; slot
// j then holds output bitrev(j)) and multiplies slot j by
// w_S^(i * bitrev(j)), w_S = e^(-2 pi i / S).  Points move between passes
// through shared memory padded by one word per 16 (per 32 at m = 14; no bank
// conflicts for any pass's pattern).  After the last pass (span 16) thread t
// holds points PT t .. PT t + PT - 1 of the spectrum in bit-reversed order;
// the spectrum of h is stored in that order with the 1/M scale folded in
// (float4 q of thread t, points PT t + 2q and PT t + 2q + 1, at index
// q*T + t, so that a warp's reads are contiguous), the product needs no
// permutation, and the inverse runs the passes backwards (conjugate
// twiddles, then the DIT G-point DFT), ending in natural order in the layout
// the input was loaded in: point t + T*j in register j, so both the input
// loads and the output stores are coalesced.  Each pass with twiddles reads
// them from its own table (two slots' twiddles per 16-byte word, by group
// position), computed in FP64 at plan time and rounded once: consecutive
// threads read consecutive words, and every point takes one complex
// multiply per pass.  Complex sums and differences are packed two-lane FP32
// instructions (real and imaginary part in one register pair).
#include "fft_core.cuh"

namespace tfx {
namespace {

// One block pair of the single-block scheme: blocks 2pr and 2pr + 1.  REV:
// input and output rows in reverse time (the transposed chain, y = R h R x,
// for the input gradient of a training step).  MSE: the training loss and
// its gradient fused into the store (FirFftArgs::loss).
// Blocks 2pr and 2pr + 1 of the single-block scheme: their channels and
// first outputs.  Coordinates in 32 bits (the host keeps nb below 2^31): one
// division for block 2pr; block 2pr + 1 is the next one in its channel or
// the first of the next channel.
struct BlockPair {
    unsigned c0, c1;
    bool live1;
    int64_t n00, n01;
};
__device__ __forceinline__ BlockPair block_pair(const FirFftArgs& a, int64_t pr) {
    const unsigned k0 = 2u * (unsigned)pr, nbpc = (unsigned)a.nbpc;
    BlockPair q;
    q.live1 = k0 + 1u < (unsigned)a.nb;
    q.c0 = k0 / nbpc;
    const unsigned r0 = k0 - q.c0 * nbpc;
    const bool wrap = r0 + 1u == nbpc;
    q.c1 = q.live1 && wrap ? q.c0 + 1u : q.c0;
    const unsigned r1 = q.live1 ? (wrap ? 0u : r0 + 1u) : 0u;
    q.n00 = (int64_t)r0 * a.B;
    q.n01 = (int64_t)r1 * a.B;
    return q;
}

template <int LOGM, bool REV = false, bool MSE = false>
__device__ __forceinline__ void fft_block_pair(const FirFftArgs& a, int64_t pr, float2* sb, int t) {
    using F = FftShape<LOGM>;
    const int Hh = a.L - 1;
    const BlockPair q = block_pair(a, pr);
    const unsigned c0 = q.c0, c1 = q.c1;
    const bool live1 = q.live1;
    const int64_t n00 = q.n00, n01 = q.n01;
    float2 v[F::PT];
    load_pair<LOGM, REV>(v, a.x + c0 * a.ldx, a.x + c1 * a.ldx, live1, n00 - Hh, n01 - Hh, a.N, t);
    forward_from<LOGM, 0>(v, a.tw, sb, t);
    // spectrum product: thread t holds positions PT t .. PT t + PT - 1,
    // stored as float4 q (positions PT t + 2q, PT t + 2q + 1) at index q*T + t
    const float4* h4 = reinterpret_cast<const float4*>(a.H) + t;
#pragma unroll
    for (int q = 0; q < F::PT / 2; ++q) {
        const float4 h = ld_tw4(h4 + q * F::T);
        v[2 * q] = cmul(v[2 * q], make_float2(h.x, h.y));
        v[2 * q + 1] = cmul(v[2 * q + 1], make_float2(h.z, h.w));
    }
    inverse_from<LOGM, F::NP - 1, last_forward_group<LOGM>()>(v, a.tw, sb, t);
    const int m0 = (int)(a.N - n00 < a.B ? a.N - n00 : a.B);
    const int m1 = live1 ? (int)(a.N - n01 < a.B ? a.N - n01 : a.B) : 0;
    if constexpr (!MSE) {
        store_pair<LOGM, REV>(v, a.y + c0 * a.ldy, a.y + c1 * a.ldy, n00, n01, a.N, Hh, m0, m1, t);
    } else {
        __shared__ double red[32];
        const float accf = store_pair_mse<LOGM>(v, a.y + c0 * a.ldy, a.y + c1 * a.ldy, a.tgt + c0 * a.ldy,
                                                a.tgt + c1 * a.ldy, a.gout + c0 * a.ldy, a.gout + c1 * a.ldy, n00,
                                                n01, Hh, m0, m1, t, a.gscale);
        // FP32 per thread, FP64 across threads (as k_mse)
        double acc = (double)accf;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((t & 31) == 0) red[t >> 5] = acc;
        __syncthreads();
        if (t == 0) {
            double sum = 0.0;
            for (int w = 0; w < FftShape<LOGM>::T / 32; ++w) sum += red[w];
            atomicAdd(a.loss, sum * a.lscale);
        }
    }
}

// Single-block overlap-save: CTA k transforms blocks 2k and 2k + 1.
template <int LOGM, bool REV, bool MSE = false>
__global__ void __launch_bounds__(FftShape<LOGM>::T, FftShape<LOGM>::MINB) k_fir_fft(FirFftArgs a) {
    extern __shared__ float2 sb[];
    fft_block_pair<LOGM, REV, MSE>(a, blockIdx.x, sb, threadIdx.x);
}

// One training step's forward on the spectral route, with the coefficient
// gradients' correlation fused in.  Persistent CTAs take block pairs pr =
// blockIdx.x, + gridDim.x, ...; for each: the forward transform X of the two
// input windows (kept in shared memory, each thread its own slots), the
// product with H and the inverse transform, the store of y with the MSE
// against the target (g = gscale (y - t) stored, the loss summed), then the
// forward transform G of the two gradient windows (zeros before the
// outputs, g at them: the registers the store left) and acc += conj(X) G.
// acc is the sum over the CTA's pairs of the block correlation spectra that
// k_chain_xcorr computes from x and g in memory (any pairing of two blocks
// as real and imaginary parts gives the same sum after the mirror step), so
// the coefficient gradients follow from part[blockIdx.x] unchanged, and x
// and g are not read again.  The loss: FP32 per thread and pair, FP64
// across pairs and threads, one FP64 atomic per CTA.
template <int LOGM>
__global__ void __launch_bounds__(FftShape<LOGM>::T, LOGM <= 12 ? 2 : 1)
    k_fir_fft_train(FirFftArgs a, float2* __restrict__ part) {
    using F = FftShape<LOGM>;
    static_assert(F::PT == 16, "spectral training transforms: 4096 and 8192 points");
    extern __shared__ float2 sb[];
    float2* zx = sb + (F::M + F::M / 16);  // X, each thread its own slots
    const int t = threadIdx.x;
    const int Hh = a.L - 1;
    float2 acc[F::PT];
#pragma unroll
    for (int j = 0; j < F::PT; ++j) acc[j] = make_float2(0.f, 0.f);
    double lsum = 0.0;
    const int64_t npairs = (a.nb + 1) / 2;
    for (int64_t pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const BlockPair q = block_pair(a, pr);
        float2 v[F::PT];
        __syncthreads();  // the previous pair's last exchange is done with sb
        load_pair<LOGM>(v, a.x + q.c0 * a.ldx, a.x + q.c1 * a.ldx, q.live1, q.n00 - Hh, q.n01 - Hh, a.N, t);
        forward_from<LOGM, 0>(v, a.tw, sb, t);
#pragma unroll
        for (int j = 0; j < F::PT; ++j) zx[j * F::T + t] = v[j];
        const float4* h4 = reinterpret_cast<const float4*>(a.H) + t;
#pragma unroll
        for (int k = 0; k < F::PT / 2; ++k) {
            const float4 h = ld_tw4(h4 + k * F::T);
            v[2 * k] = cmul(v[2 * k], make_float2(h.x, h.y));
            v[2 * k + 1] = cmul(v[2 * k + 1], make_float2(h.z, h.w));
        }
        inverse_from<LOGM, F::NP - 1, last_forward_group<LOGM>()>(v, a.tw, sb, t);
        const int m0 = (int)(a.N - q.n00 < a.B ? a.N - q.n00 : a.B);
        const int m1 = q.live1 ? (int)(a.N - q.n01 < a.B ? a.N - q.n01 : a.B) : 0;
        lsum += (double)store_pair_mse<LOGM, true>(v, a.y + q.c0 * a.ldy, a.y + q.c1 * a.ldy, a.tgt + q.c0 * a.ldy,
                                                   a.tgt + q.c1 * a.ldy, a.gout + q.c0 * a.ldy,
                                                   a.gout + q.c1 * a.ldy, q.n00, q.n01, Hh, m0, m1, t, a.gscale);
        __syncthreads();  // the inverse's last exchange is done with sb
        forward_from<LOGM, 0>(v, a.tw, sb, t);
#pragma unroll
        for (int j = 0; j < F::PT; ++j) {
            const float2 w = zx[j * F::T + t];
            acc[j].x = fmaf(v[j].x, w.x, fmaf(v[j].y, w.y, acc[j].x));
            acc[j].y = fmaf(v[j].y, w.x, fmaf(-v[j].x, w.y, acc[j].y));
        }
    }
    float4* out = reinterpret_cast<float4*>(part + (int64_t)blockIdx.x * F::M) + t;
#pragma unroll
    for (int k = 0; k < F::PT / 2; ++k)
        out[k * F::T] = make_float4(acc[2 * k].x, acc[2 * k].y, acc[2 * k + 1].x, acc[2 * k + 1].y);
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((t & 31) == 0) red[t >> 5] = lsum;
    __syncthreads();
    if (t == 0) {
        double sum = 0.0;
        for (int w = 0; w < F::T / 32; ++w) sum += red[w];
        atomicAdd(a.loss, sum * a.lscale);
    }
}

// Single-block overlap-save over many clips in one launch (a batch of
// composed chains sharing one transform size): CTA k maps to its clip by a
// binary search over the clips' block-pair prefix sums, then transforms that
// clip's block pair k - prefix[clip] with the clip's own spectrum.  The
// clip of every CTA is precomputed on the host (unit_of[k], one load
// instead of a serial binary search over the prefix sums).
template <int LOGM>
__global__ void __launch_bounds__(FftShape<LOGM>::T, FftShape<LOGM>::MINB)
    k_fir_fft_batched(const BatchFft* __restrict__ units, const int64_t* __restrict__ prefix,
                      const int32_t* __restrict__ unit_of, BatchBases bases, const float2* __restrict__ tw) {
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    const int64_t k = blockIdx.x;
    const int u = __ldg(unit_of + k);
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
// like H: float4 q of thread t (positions PT t + 2q, PT t + 2q + 1) at q*T + t.
template <int LOGM>
__global__ void __launch_bounds__(FftShape<LOGM>::T, FftShape<LOGM>::MINB) k_fir_fft_spec(FirFftArgs a) {
    using F = FftShape<LOGM>;
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    const int64_t pb = blockIdx.x;
    const unsigned r = blockIdx.x / (unsigned)a.nbpc, b = blockIdx.x - r * (unsigned)a.nbpc;
    const int64_t c0 = 2 * (int64_t)r;
    const bool live1 = c0 + 1 < a.C;
    const float* x0 = a.x + c0 * a.ldx;
    const int64_t s0 = ((int64_t)b - 1) * a.B;
    float2 v[F::PT];
    load_pair<LOGM>(v, x0, live1 ? x0 + a.ldx : x0, live1, s0, s0, a.N, t);
    forward_from<LOGM, 0>(v, a.tw, sb, t);
    float4* z = reinterpret_cast<float4*>(a.Z + pb * F::M) + t;
#pragma unroll
    for (int q = 0; q < F::PT / 2; ++q) z[q * F::T] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
}

// Partitioned overlap-save, step 2: block b of a channel pair is the inverse
// transform of sum over partitions p <= b of H_p Z_(b-p) (h split into P
// partitions of B taps, h_p[k] = h[pB + k]), whose last B points are outputs
// [bB, (b + 1) B).
template <int LOGM>
__global__ void __launch_bounds__(FftShape<LOGM>::T, FftShape<LOGM>::MINB) k_fir_fft_conv(FirFftArgs a) {
    using F = FftShape<LOGM>;
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    const int64_t pb = blockIdx.x;
    const unsigned r = blockIdx.x / (unsigned)a.nbpc, b = blockIdx.x - r * (unsigned)a.nbpc;
    const int64_t c0 = 2 * (int64_t)r;
    const bool live1 = c0 + 1 < a.C;
    float2 v[F::PT];
#pragma unroll
    for (int j = 0; j < F::PT; ++j) v[j] = make_float2(0.f, 0.f);
    const int np = (int)b + 1 < a.P ? (int)b + 1 : a.P;
    for (int p = 0; p < np; ++p) {
        const float4* h4 = reinterpret_cast<const float4*>(a.H + (int64_t)p * F::M) + t;
        const float4* z4 = reinterpret_cast<const float4*>(a.Z + (pb - p) * F::M) + t;
#pragma unroll
        for (int q = 0; q < F::PT / 2; ++q) {
            const float4 h = __ldg(h4 + q * F::T), z = __ldg(z4 + q * F::T);
            v[2 * q].x = fmaf(z.x, h.x, fmaf(-z.y, h.y, v[2 * q].x));
            v[2 * q].y = fmaf(z.x, h.y, fmaf(z.y, h.x, v[2 * q].y));
            v[2 * q + 1].x = fmaf(z.z, h.z, fmaf(-z.w, h.w, v[2 * q + 1].x));
            v[2 * q + 1].y = fmaf(z.z, h.w, fmaf(z.w, h.z, v[2 * q + 1].y));
        }
    }
    inverse_from<LOGM, F::NP - 1>(v, a.tw, sb, t);
    const int64_t n0 = (int64_t)b * a.B;
    const int m0 = (int)(a.N - n0 < a.B ? a.N - n0 : a.B);
    float* y0 = a.y + c0 * a.ldy;
    store_pair<LOGM>(v, y0, live1 ? y0 + a.ldy : y0, n0, n0, a.N, F::M - a.B, m0, live1 ? m0 : 0, t);
}

// Spectrum of a FIR (or of each of its P partitions of B taps) computed on
// the device from FP64 taps, for coefficient updates without a host round
// trip: CTA p transforms h[pB, pB + len) (len = B, or L when P = 0) zero-
// padded to M points with the same forward transform the filter uses, and
// stores it as the filter reads it: scaled by 1/M, bit-reversed, float4 q of
// thread t at q*T + t.
template <int LOGM>
__global__ void __launch_bounds__(FftShape<LOGM>::T, FftShape<LOGM>::MINB)
    k_fir_fft_spectrum(const double* __restrict__ taps, int L, int B, int P, const float2* __restrict__ tw,
                       float2* __restrict__ H) {
    using F = FftShape<LOGM>;
    extern __shared__ float2 sb[];
    const int t = threadIdx.x;
    const int part = blockIdx.x;
    const int64_t first = P > 0 ? (int64_t)part * B : 0;
    const int len = P > 0 ? B : L;
    float2 v[F::PT];
#pragma unroll
    for (int j = 0; j < F::PT; ++j) {
        const int n = t + F::T * j;
        const int64_t k = first + n;
        v[j] = make_float2(n < len && k < L ? (float)taps[k] : 0.f, 0.f);
    }
    forward_from<LOGM, 0>(v, tw, sb, t);
    const float inv = 1.0f / (float)F::M;
    float4* h4 = reinterpret_cast<float4*>(H + (int64_t)part * F::M) + t;
#pragma unroll
    for (int q = 0; q < F::PT / 2; ++q)
        h4[q * F::T] = make_float4(v[2 * q].x * inv, v[2 * q].y * inv, v[2 * q + 1].x * inv, v[2 * q + 1].y * inv);
}

template <int LOGM>
cudaError_t launch_spectrum_log(const double* taps, int L, int B, int P, const float2* tw, float2* H,
                                cudaStream_t s) {
    constexpr int T = FftShape<LOGM>::T;
    const size_t smem = fir_fft_smem_bytes(1 << LOGM);
    k_fir_fft_spectrum<LOGM><<<(unsigned)(P > 0 ? P : 1), T, smem, s>>>(taps, L, B, P, tw, H);
    return cudaGetLastError();
}

template <int LOGM>
cudaError_t launch_log(const FirFftArgs& a, cudaStream_t s) {
    constexpr int T = FftShape<LOGM>::T;
    const size_t smem = fir_fft_smem_bytes(1 << LOGM);
    if (a.P == 0) {
        if (a.loss && a.rev) return cudaErrorInvalidValue;
        if (a.loss)
            k_fir_fft<LOGM, false, true><<<(unsigned)((a.nb + 1) / 2), T, smem, s>>>(a);
        else if (a.rev)
            k_fir_fft<LOGM, true><<<(unsigned)((a.nb + 1) / 2), T, smem, s>>>(a);
        else
            k_fir_fft<LOGM, false><<<(unsigned)((a.nb + 1) / 2), T, smem, s>>>(a);
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
    cudaError_t e = cudaFuncSetAttribute(k_fir_fft<LOGM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft<LOGM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft<LOGM, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft_spec<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft_conv<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft_spectrum<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fir_fft_batched<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (LOGM == 12 || LOGM == 13)
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fir_fft_train<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)xcorr_smem_bytes(1 << LOGM));
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
cudaError_t launch_batched_log(const BatchFft* units, const int64_t* prefix, const int32_t* unit_of, int64_t ctas,
                               BatchBases bases, const float2* tw, cudaStream_t s) {
    constexpr int T = FftShape<LOGM>::T;
    const size_t smem = fir_fft_smem_bytes(1 << LOGM);
    k_fir_fft_batched<LOGM><<<(unsigned)ctas, T, smem, s>>>(units, prefix, unit_of, bases, tw);
    return cudaGetLastError();
}

cudaError_t launch_fir_fft_batched(int m, const BatchFft* units, const int64_t* prefix, const int32_t* unit_of,
                                   int nunits, int64_t ctas, BatchBases bases, const float2* tw, cudaStream_t s) {
    if (ctas <= 0 || nunits <= 0) return cudaSuccess;
    switch (m) {
        case 10: return launch_batched_log<10>(units, prefix, unit_of, ctas, bases, tw, s);
        case 11: return launch_batched_log<11>(units, prefix, unit_of, ctas, bases, tw, s);
        case 12: return launch_batched_log<12>(units, prefix, unit_of, ctas, bases, tw, s);
        case 13: return launch_batched_log<13>(units, prefix, unit_of, ctas, bases, tw, s);
        case 14: return launch_batched_log<14>(units, prefix, unit_of, ctas, bases, tw, s);
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
    if (a.nb > INT32_MAX || (a.P > 0 && (a.C + 1) / 2 * a.nbpc > INT32_MAX)) return cudaErrorInvalidValue;
    if (a.loss && a.P > 0) return cudaErrorInvalidValue;  // the fused loss is single-block only
    switch (a.m) {
        case 10: return launch_log<10>(a, s);
        case 11: return launch_log<11>(a, s);
        case 12: return launch_log<12>(a, s);
        case 13: return launch_log<13>(a, s);
        case 14: return launch_log<14>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fir_fft_train(const FirFftArgs& a, float2* part, int grid, cudaStream_t s) {
    if (a.P != 0 || a.rev || !a.loss || !a.tgt || !a.gout || (a.nb + 1) / 2 > INT32_MAX || grid < 1)
        return cudaErrorInvalidValue;
    switch (a.m) {
        case 12:
            k_fir_fft_train<12><<<(unsigned)grid, FftShape<12>::T, xcorr_smem_bytes(4096), s>>>(a, part);
            break;
        case 13:
            k_fir_fft_train<13><<<(unsigned)grid, FftShape<13>::T, xcorr_smem_bytes(8192), s>>>(a, part);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace tfx
