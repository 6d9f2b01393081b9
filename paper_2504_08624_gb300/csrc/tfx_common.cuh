// Internal definitions shared by the libtfx kernels and the host plan code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tfx.h"

namespace tfx {

// CTA shape of the scan / fused kernels: NT threads, each owning a contiguous
// chunk of T samples, so one tile is NT*T samples of one channel.
constexpr int NT = 256;
constexpr int NWARP = NT / 32;
constexpr int T_CHUNK = 32;
constexpr int TILE = NT * T_CHUNK;  // 8192 samples
// Cascade-only units (no FIR) run 128-thread CTAs with 64 samples per thread
// (the same 8192-sample tile): fewer scan steps and barriers per sample.
constexpr int NT_CASCADE = 128;
constexpr int T_CASCADE = 64;
static_assert(NT_CASCADE * T_CASCADE == TILE, "cascade tile must match the fused tile");
// FIR register blocking: each thread produces FIR_R consecutive outputs per
// pass and walks the taps FIR_R at a time.
constexpr int FIR_R = 16;
// Entries per section in the chunk-transfer power table: A^k, k = 0..1024.
constexpr int PW_LEN = 1025;
// Zero padding in front of the FIR window (shared memory), >= 2*FIR_R.
constexpr int FIR_PAD = 32;
// Device-side bounded waits give up after this long and record TFX_ERR_TIMEOUT.
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

// Points each thread holds in the register-resident FFT of M = 2^m points
// (host and device agree on it: it fixes the spectra's storage order): 16,
// or 32 for 16384 points (512 threads, radix-32 passes).
__host__ __device__ constexpr int fft_pt(int m) { return m == 14 ? 32 : 16; }

// Per-unit device constants (one "unit" = an optional SOS cascade followed
// by an optional FIR; consecutive SOS stages are merged into one cascade).
struct UnitConst {
    int S;             // sections
    int L;             // FIR taps (0 = no FIR)
    int H;             // FIR halo = L - 1 (0 without FIR)
    int nkb;           // FIR tap blocks of FIR_R (taps zero-padded to nkb*FIR_R)
    float gain;        // output scale when the unit ends without an FIR
    const float* coef; // [S][8]: b0 c1 c2 a1 a2 (a0-normalised; c1 = b1 - a1 b0, c2 = b2 - a2 b0)
    const float4* pw;  // [S][PW_LEN]: A^k, A = chunk transfer matrix (row-major 2x2)
    const float* taps; // [nkb*FIR_R] FP32 taps, zero-padded
    const double4* pw64;  // cascades with a pole of radius > 0.999: the same powers in FP64, else null
};

// Look-back carry of one (tile, section): a 2-vector published with a status
// (0 = nothing yet, 1 = tile aggregate, 2 = inclusive prefix).  Stored as two
// 8-byte halves {status, x} and {status, y}; each half is single-copy atomic,
// and a reader accepts the word only when both halves carry the same status.
struct __align__(16) Carry {
    unsigned fx;
    float x;
    unsigned fy;
    float y;
};

// Scratch for one execution of one unit (inside the caller's workspace).
struct UnitScratch {
    unsigned* ticket;   // tile ticket counter (reset per execution)
    unsigned* flags;    // [tiles]: FIR-input tail published (reset per execution)
    Carry* carry;       // [tiles][S] look-back carries (reset per execution)
    float* tails;       // [tiles][tail_len]: last FIR-input samples of each tile
    int tail_len;       // min(H, TILE)
};

struct UnitArgs {
    const float* x;
    float* y;
    int64_t ldx, ldy;
    int64_t C, N;
    int64_t ntt;  // time tiles per channel
    UnitConst k;
    UnitScratch sc;
    int* status;     // device status word (TFX_OK or TFX_ERR_TIMEOUT)
    int64_t drop_tile;  // test hook: this tile never publishes (-1 = off)
    // training forward (warp-tile cascade only): the true state of every
    // section at every 32-sample chunk start, [C][S][nch] float2, or null
    float2* ckpt;
    int64_t nch;
};

// Batched execution: buffer pointers of a batch descriptor are offsets into
// one of three bases (0: the packed batch input, 1: the packed batch output,
// 2: the workspace).
struct BatchBases {
    const float* x;
    float* y;
    float* ws;
    __device__ __forceinline__ float* ptr(int sel) const {
        return sel == 0 ? const_cast<float*>(x) : (sel == 1 ? y : ws);
    }
};

struct BatchUnit {
    UnitArgs a;          // constants, sizes, status; x, y, scratch filled in from the offsets below
    int x_sel, y_sel;    // bases for x and y
    int64_t x_off, y_off;                 // in floats
    int64_t flags_off, carry_off, tails_off;  // in bytes, into the workspace
};

// Reverse-time adjoint of an SOS cascade (warp-tile geometry of the forward
// training pass: 32 lanes x T_CHUNK samples per tile).
struct BwdArgs {
    const float* u0;   // the cascade's forward input, row stride ldu
    int64_t ldu;
    const float* g;    // dL/d(cascade output), row stride ldg
    int64_t ldg;
    int g_rev;         // 1: row holds the gradient time-reversed (sample n at N-1-n)
    float* gout;       // dL/d(cascade input), row stride ldo (null: not written)
    int64_t ldo;
    int out_rev;       // 1: write gout time-reversed
    const float2* ckpt;  // [C][S][nch] forward chunk-start states
    int64_t nch;
    int64_t C, N, ntt;   // ntt = tiles of 32 * T_CHUNK samples per channel
    UnitConst k;         // coef rows [S][8]: b0 c1 c2 a1 a2 d (d = a1 b2 - a2 b1)
    unsigned* ticket;
    Carry* carry;        // [tiles][S] reverse look-back carries
    float* part;         // [S * 5][tiles]: per-tile partial dL/d(b0 b1 b2 a1 a2), column-major
    int* status;
};

// Operand precision of the tensor-core FIR.
enum { FIR_TC_FP16_SPLIT = 0, FIR_TC_BF16_SPLIT = 1, FIR_TC_BF16_PLAIN = 2 };

// Tensor-core FIR (Toeplitz-block GEMM) launch arguments.
struct FirTcArgs {
    const float* x;
    float* y;
    int64_t ldx, ldy;
    int64_t C, N;
    int64_t ntt;      // tiles per channel (128 * NB output samples each)
    int L;            // taps
    int W;            // L - 1 rounded up to a multiple of 16
    int nK;           // K-steps of 16: (W + 128) / 16
    int NB;           // output blocks of 128 samples per tile (MMA N)
    int rows;         // rows of the shared-memory signal window grid
    int tmem_cols;    // TMEM columns allocated (power of two >= NB)
    int a_chunks;     // 16-byte chunks per tap table = 2 * nK + 16
    int mode;         // FIR_TC_FP16_SPLIT, FIR_TC_BF16_SPLIT or FIR_TC_BF16_PLAIN
    int persistent;   // 0: one tile per CTA; 1: persistent, resident taps, 2-stage windows;
                      // 2: persistent, taps streamed in K-blocks, single window
    int grid;         // persistent grid size (one CTA per SM)
    float tap_unscale;  // 1 / (power-of-two scale applied to the FP16 taps)
    const uint4* a_hi;  // [a_chunks][8 copies] high parts of the shifted (scaled) taps
    const uint4* a_lo;  // same, low parts
    int* status;
};

// Cascade on the tensor cores by channel segments (k_sos_tc).
// Blocks of TCS_KB samples; per block, one M = 128 GEMM row set gives the
// TCS_KB outputs of the block's zero-state response (lower-triangular
// Toeplitz of the cascade's impulse response) and the 16 components of its
// zero-start end state; a 16-dimensional scan over blocks gives each block's
// start state s_b, and a K = 16 GEMM adds the free response O s_b.
constexpr int SEG_SMAX = 8;                  // sections (state dimension 2S <= 16)
constexpr int TCS_KB = 112;                  // samples per block (M rows 0..111; 112..127: end state)
constexpr int TCS_NB = 128;                  // blocks per tile (N)
constexpr int TCS_TILE = TCS_KB * TCS_NB;    // 14336 samples
constexpr int TCS_A1_BYTES = 128 * TCS_KB * 2;  // one 16-bit [128 x 112] operand, canonical K-major
constexpr int TCS_A2_BYTES = 128 * 16 * 2;      // one 16-bit [128 x 16] operand
struct SegArgs {
    const float* x;
    float* y;
    int64_t ldx, ldy;
    int64_t C, N;
    int S;
    float gain;
    const float* coef;  // [S][8] as UnitConst::coef
    int64_t Lseg;       // segment length, a multiple of TCS_TILE
    int64_t P;          // segments per channel
    int D;              // warm-up samples run before every segment but a channel's first (multiple of TCS_KB)
    // tensor-core segment kernel
    const uint4* a1;       // [2][TCS_A1_BYTES / 16]: [Toeplitz rows; end-state rows], hi then lo (FP16, row-scaled)
    const uint4* a2;       // [2][TCS_A2_BYTES / 16]: free-response rows O, hi then lo (same row scales)
    const float* rowinv;   // [128]: 1 / row scale
    const float* phib;     // [8][16][16]: (A^TCS_KB)^j, j = 1..8 (block transfer powers)
    int* status;
};

// FIR by FFT overlap-save: blocks of B = M - (L - 1) outputs, two blocks per CTA.
struct FirFftArgs {
    const float* x;
    float* y;
    int64_t ldx, ldy;
    int64_t C, N;
    int L;
    int M, m;          // FFT size M = 2^m (complex points)
    int B;             // outputs per block
    int64_t nbpc, nb;  // blocks per channel, blocks in all
    const float2* H;   // [max(P,1)][M] spectra of h (or of its partitions), bit-reversed order, scaled by 1/M
    const float2* tw;  // per-pass twiddle tables (see k_fir_fft.cu)
    int P;             // 0: single-block overlap-save; else partitions of B = M/2 taps
    float2* Z;         // partitioned: [ceil(C/2)][nbpc][M] segment spectra (workspace)
    int rev;           // single-block: rows of x and y in reverse time (the transposed filter)
    // single-block, forward time: the MSE against tgt fused into the store
    // (rows with stride ldy): gout = gscale (y - tgt), and the sum of
    // (y - tgt)^2 times lscale added into *loss (one FP64 atomic per CTA);
    // loss == nullptr: plain filter
    const float* tgt;
    float* gout;
    double* loss;
    float gscale;
    double lscale;
};

// One composed clip of a batch (the whole chain as one FFT FIR): where its
// samples are, its shape and block geometry, its spectrum.
struct BatchFft {
    int x_sel, y_sel;
    int64_t x_off, y_off;  // in floats
    int64_t C, N;
    int L, B;
    int64_t nbpc, nb;
    const float2* H;
};

// Sections a spectral training plan takes (all its cascades together).
constexpr int SPEC_SMAX = 16;

// Block correlation spectra of a training step (k_spectral.cu): channel
// pairs x blocks of B gradient samples against input windows of J + B.
struct XcorrArgs {
    const float* x;
    const float* g;
    int64_t ldx, ldg;
    int64_t C, N;
    int J, B;             // lags kept (the composite response's halo) and gradient samples per block
    int64_t nbpc, items;  // blocks per channel; channel pairs x blocks
    const float2* tw;
    float2* part;         // [grid][M] partial spectra (storage layout)
};

struct BatchFir {
    FirTcArgs a;           // x and y filled in from the offsets below
    int x_sel, y_sel;
    int64_t x_off, y_off;  // in floats
};

// ---------------------------------------------------------------------------
// device helpers

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ float4 ld_relaxed_f4(const float4* p) {
    float4 v;
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

// Wait until *flag >= want.  Returns the flag value, or 0 if the wait gave up
// (time limit reached, or another CTA already recorded an error), in which
// case the status word holds TFX_ERR_TIMEOUT and the caller continues with
// zero data so that every CTA still terminates.
__device__ __forceinline__ unsigned wait_flag(const unsigned* flag, unsigned want, int* status) {
    unsigned v = ld_acquire_u32(flag);
    if (v >= want) return v;
    unsigned long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
        v = ld_acquire_u32(flag);
        if (v >= want) return v;
        if (*(volatile int*)status != 0) return 0;
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            atomicCAS(status, 0, (int)TFX_ERR_TIMEOUT);
            return 0;
        }
    }
}

__device__ __forceinline__ void publish_carry(Carry* p, unsigned status, float2 v) {
    asm volatile("st.relaxed.gpu.global.v4.b32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(status),
                 "r"(__float_as_uint(v.x)), "r"(status), "r"(__float_as_uint(v.y))
                 : "memory");
}

// Status of a carry and its value (0 while nothing is published).
__device__ __forceinline__ unsigned read_carry(const Carry* p, float2& v) {
    for (;;) {
        unsigned fx, x, fy, y;
        asm volatile("ld.relaxed.gpu.global.v4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(fx), "=r"(x), "=r"(fy), "=r"(y)
                     : "l"(p)
                     : "memory");
        if (fx == fy) {
            v = make_float2(__uint_as_float(x), __uint_as_float(y));
            return fx;
        }
    }
}

// Wait (bounded, like wait_flag) until a carry has status >= 1.
__device__ __forceinline__ unsigned wait_carry(const Carry* p, float2& v, int* status) {
    unsigned f = read_carry(p, v);
    if (f >= 1u) return f;
    unsigned long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        f = read_carry(p, v);
        if (f >= 1u) return f;
        if (*(volatile int*)status != 0) return 0;
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            atomicCAS(status, 0, (int)TFX_ERR_TIMEOUT);
            return 0;
        }
    }
}

// FP64 carries (cascades with a pole of radius > 0.999): the same 16-byte
// word, two doubles whose two lowest mantissa bits hold the status (a
// perturbation of 2^-51 relative, far below the FP32 data).
__device__ __forceinline__ void publish_carry64(Carry* p, unsigned status, double2 v) {
    const unsigned long long x = (__double_as_longlong(v.x) & ~3ull) | status;
    const unsigned long long y = (__double_as_longlong(v.y) & ~3ull) | status;
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1,%2};" ::"l"(p), "l"(x), "l"(y) : "memory");
}

__device__ __forceinline__ unsigned read_carry64(const Carry* p, double2& v) {
    for (;;) {
        unsigned long long x, y;
        asm volatile("ld.relaxed.gpu.global.v2.b64 {%0,%1}, [%2];" : "=l"(x), "=l"(y) : "l"(p) : "memory");
        if ((x & 3ull) == (y & 3ull)) {
            v = make_double2(__longlong_as_double((long long)(x & ~3ull)), __longlong_as_double((long long)(y & ~3ull)));
            return (unsigned)(x & 3ull);
        }
    }
}

__device__ __forceinline__ unsigned wait_carry64(const Carry* p, double2& v, int* status) {
    unsigned f = read_carry64(p, v);
    if (f >= 1u) return f;
    unsigned long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        f = read_carry64(p, v);
        if (f >= 1u) return f;
        if (*(volatile int*)status != 0) return 0;
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            atomicCAS(status, 0, (int)TFX_ERR_TIMEOUT);
            return 0;
        }
    }
}

__device__ __forceinline__ double2 mv2d(double4 m, double2 v) {
    return make_double2(fma(m.x, v.x, m.y * v.y), fma(m.z, v.x, m.w * v.y));
}
__device__ __forceinline__ double4 mm2d(double4 a, double4 b) {
    return make_double4(fma(a.x, b.x, a.y * b.z), fma(a.x, b.y, a.y * b.w), fma(a.z, b.x, a.w * b.z),
                        fma(a.z, b.y, a.w * b.w));
}

// 2x2 row-major matrix (float4 = m00 m01 m10 m11) helpers
__device__ __forceinline__ float2 mv2(float4 m, float2 v) {
    return make_float2(fmaf(m.x, v.x, m.y * v.y), fmaf(m.z, v.x, m.w * v.y));
}
__device__ __forceinline__ float4 mm2(float4 a, float4 b) {
    return make_float4(fmaf(a.x, b.x, a.y * b.z), fmaf(a.x, b.y, a.y * b.w),
                       fmaf(a.z, b.x, a.w * b.z), fmaf(a.z, b.y, a.w * b.w));
}

// Launchers (defined in the kernel translation units).
cudaError_t launch_unit(const UnitArgs& a, cudaStream_t s);
cudaError_t launch_sos_tc(const SegArgs& a, int grid, cudaStream_t s);
cudaError_t prepare_sos_tc();
size_t sos_tc_smem_bytes();
cudaError_t launch_sos_warp(const UnitArgs& a, cudaStream_t s);
cudaError_t launch_plain_sos(const float* x, float* y, int64_t C, int64_t N, int64_t ldx,
                             int64_t ldy, int S, const float* coef, cudaStream_t s);
cudaError_t launch_plain_fir(const float* x, float* y, int64_t C, int64_t N, int64_t ldx,
                             int64_t ldy, int L, const float* taps, cudaStream_t s);
cudaError_t launch_copy_rows(const float* x, float* y, int64_t C, int64_t N, int64_t ldx,
                             int64_t ldy, cudaStream_t s);
size_t unit_smem_bytes(const UnitConst& k);
size_t fir_tc_smem_bytes(const FirTcArgs& a);
cudaError_t prepare_fir_tc(size_t smem);
cudaError_t prepare_fir_tc_ws(size_t smem);
cudaError_t prepare_fir_tc_long(size_t smem);
size_t fir_tc_long_smem(int rows);
constexpr int TC_KBLK = 64;  // K-steps per streamed tap block
cudaError_t launch_fir_tc(const FirTcArgs& a, cudaStream_t s);
size_t fir_fft_smem_bytes(int M);
cudaError_t prepare_fir_fft(int M);
cudaError_t launch_fir_fft(const FirFftArgs& a, cudaStream_t s);
// spectral training step: forward + MSE + the correlation partials, one CTA
// per part[] row (k_fir_fft_train)
cudaError_t launch_fir_fft_train(const FirFftArgs& a, float2* part, int grid, cudaStream_t s);
size_t xcorr_smem_bytes(int M);
int xcorr_ctas_per_sm(int m);
cudaError_t prepare_spectral(int m);
cudaError_t launch_chain_xcorr(int m, const XcorrArgs& a, int grid, cudaStream_t s);
cudaError_t launch_xcorr_reduce(const float2* part, int G, int M, double2* P, cudaStream_t s);
// zt: e^(-2 pi i k / M) for bins k < M (FP64, plan constant).
cudaError_t launch_chain_spectrum(const double* raw, int S, const float2* Hf, const double2* zt, int m, float2* H,
                                  cudaStream_t s);
cudaError_t launch_chain_tail(int m, const float2* H, const float2* tw, int J, int* status, cudaStream_t s);
// Scratch of launch_chain_grads: the blocks' partial sums of the section
// gradients, which launch_spectral_finalize adds up and maps to the raw rows
// (dcoef at dst[s] for section s).
size_t chain_grads_scratch_bytes(int m, int S);
cudaError_t launch_chain_grads(int m, const double2* P, const double* raw, int S, const float2* Hf,
                               const double2* zt, const float2* tw, int L, void* scratch, float2* wfir, double* dh,
                               cudaStream_t s);
cudaError_t launch_spectral_finalize(int m, const void* scratch, int S, const double* raw, const int64_t* dst,
                                     double* dcoef, cudaStream_t s);
cudaError_t launch_fir_fft_batched(int m, const BatchFft* units, const int64_t* prefix, const int32_t* unit_of,
                                   int nunits, int64_t ctas, BatchBases bases, const float2* tw, cudaStream_t s);
cudaError_t launch_fir_fft_spectrum(const double* taps, int L, int M, int B, int P, const float2* tw, float2* H,
                                    cudaStream_t s);
cudaError_t launch_fir_tc_batched(const BatchFir* units, const int64_t* prefix, int nunits, int64_t tiles,
                                  BatchBases bases, size_t smem, cudaStream_t s);
cudaError_t prepare_fir_tc_batched(size_t smem);
cudaError_t prepare_unit(const UnitConst& k);
cudaError_t launch_unit_batched(bool has_fir, const BatchUnit* units, const int64_t* prefix, int nunits,
                                int64_t tiles, unsigned* ticket, BatchBases bases, size_t smem, cudaStream_t s);
cudaError_t prepare_unit_batched(size_t smem);

// Backward (adjoint) launchers, defined in k_bwd.cu.
constexpr int BWD_SMAX = 8;  // sections per cascade unit in a trainable plan
size_t sos_bwd_smem_bytes(int S);
cudaError_t prepare_sos_bwd(int S);
cudaError_t launch_sos_bwd(const BwdArgs& a, cudaStream_t s);
cudaError_t launch_flip_rows(const float* x, float* y, int64_t C, int64_t N, int64_t ldx, int64_t ldy,
                             cudaStream_t s);
constexpr int DH_BLOCK = 2048;  // samples per warp in the CUDA-core FIR tap-gradient kernel
constexpr int DH_WIN = 256;     // lags per shared-memory window
int64_t fir_dh_rows(int64_t C, int64_t N);
cudaError_t launch_fir_dh(const float* g, int64_t ldg, int g_rev, const float* u, int64_t ldu, int64_t C,
                          int64_t N, int L, int Lp, float* part, cudaStream_t s);
// Tensor-core FIR tap gradient (k_fir_dh_tc.cu): partials [L][G], G K-range CTAs.
void fir_dh_tc_geometry(int64_t C, int64_t N, int L, int sm_count, int* G, int* nwin, int* LW, int* NQ);
size_t fir_dh_tc_smem(int NQ);
cudaError_t prepare_fir_dh_tc();
cudaError_t launch_fir_dh_tc(const float* g, int64_t ldg, int g_rev, const float* u, int64_t ldu, float* gflip,
                             int64_t C, int64_t N, int L, int sm_count, float* part, int* status, cudaStream_t s);
// FP64 sums of column-major FP32 partials [ncol][rows] -> out[ncol]
cudaError_t launch_colsum(const float* part, int64_t rows, int ncol, double* out, cudaStream_t s);
cudaError_t launch_sos_grad_finalize(const double* sums, int S, const double* raw, const int64_t* dst,
                                     double* dcoef, cudaStream_t s);
cudaError_t launch_mse(const float* y, const float* t, float* g, int64_t C, int64_t N, int64_t ld,
                       double* loss, cudaStream_t s);

}  // namespace tfx
