// Plan internals shared by the plan code (plan.cu) and the batched launch
// (batch.cu): a chain grouped into units, their device constants and the
// workspace layout.  Not part of the C ABI.
#pragma once

#include <vector>

#include "tfx_common.cuh"

namespace tfx {

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct HostUnit {
    int S = 0;                  // sections
    int L = 0;                  // FIR taps (0 = none)
    std::vector<double> sec;    // [S][5] a0-normalised b0 b1 b2 a1 a2
    std::vector<double> taps;   // [L]
    // device constants (offsets into the plan's constant blob)
    size_t off_coef = 0, off_pw = 0, off_taps = 0;
    int nkb = 0;
    int64_t ntt = 0;            // time tiles per channel
    int tail_len = 0;
    // scratch sizes (bytes)
    size_t flags_bytes = 0, vals_bytes = 0, tails_bytes = 0;
    // FIR on the tensor cores (Toeplitz-block GEMM); such a unit has S == 0
    bool tc = false;
    int W = 0, nK = 0, NB = 0, rows = 0, tmem_cols = 0, a_chunks = 0;
    size_t off_ahi = 0, off_alo = 0, tc_smem = 0;
    int tc_mode = 0;
    float tap_unscale = 1.0f;
    int tc_variant = 0;  // 0: one tile per CTA, 1: persistent resident taps, 2: persistent streamed taps
    size_t tc_smem_ws = 0;
    // cascade without an FIR: warp-per-tile scan (tiles of 32 * T_CHUNK samples)
    bool warp = false;
    // a section with a pole of radius > 0.999: warp-tile scan with FP64
    // cross-tile carries and an FP64 copy of the power table
    bool hiq = false;
    size_t off_pw64 = 0;
    // FIR by FFT overlap-save (TFX_PLAN_FIR_FFT)
    bool fft = false;
    int fft_M = 0, fft_m = 0, fft_B = 0;
    int fft_P = 0;  // 0: single-block overlap-save; else partitions of fft_B = M/2 taps
    // cascade on the tensor cores by channel segments (k_sos_tc): segments per
    // channel, their length, warm-up length
    bool seg = false;
    int64_t seg_P = 0, seg_len = 0;
    int seg_D = 0;  // warm-up samples before every segment but a channel's first
    size_t off_tc = 0;
    std::vector<uint8_t> tc_a1, tc_a2;       // GEMM operands (hi, lo), canonical FP16 layout
    std::vector<float> tc_rowinv, tc_phib;   // 1 / row scales, block transfer A^112
    size_t off_H = 0, off_tw = 0;
    // trainable plans: where each section's raw row (6 values) and the FIR's
    // taps sit in the flat coefficient-gradient array, the raw rows for the
    // a0 chain rule, and the unit's saved activations
    std::vector<int64_t> dst;   // [S]
    std::vector<double> raw;    // [S][6]
    int64_t fir_dst = 0;
    size_t off_raw = 0, off_dst = 0;  // constant blob
    size_t off_act = 0;               // saved: this unit's input (units after the first)
    size_t off_ckpt = 0;              // saved: chunk-start states [C][S][nch] (cascade units)
    int Lp = 0;                       // FIR taps rounded up to 16
};

constexpr int WARP_TILE = 32 * T_CHUNK;

// Taps at or above this count go to the tensor cores (unless disabled or
// overridden per plan).
constexpr int TC_MIN_TAPS = 64;
// FIRs from this many taps run by FFT overlap-save unless the plan asks for
// the tensor cores: measured faster on GB300 at every length from 65 taps
// (16 x 2.88M samples: 104 us against 120 us at 65 taps, 144 against 209 at
// 1025); shorter FIRs stay on the CUDA cores.
constexpr int FFT_MIN_TAPS = 64;
constexpr size_t SMEM_MAX = 227 * 1024;

struct PlainStage {
    int kind;  // TFX_STAGE_FIR / TFX_STAGE_SOS
    int n;
    size_t off;  // FP32 coefficients in the constant blob (SOS: [n][8]; FIR: [n])
};

}  // namespace tfx

struct tfx_plan {
    int64_t C = 0, N = 0, ld = 0;
    uint32_t flags = 0;
    std::vector<tfx::HostUnit> units;
    std::vector<tfx::PlainStage> plain;
    char* dconst = nullptr;
    int* dstatus = nullptr;
    // workspace layout
    size_t scratch_hdr = 0;    // ticket + tail flags + carries (memset per unit execution)
    size_t scratch_bytes = 0;  // header + tails
    size_t buf_bytes = 0;      // one intermediate [C x N] buffer
    size_t ws_fused = 0, ws_plain = 0;
    int sm_count = 1;  // persistent grid size
    // trainable plans
    bool train = false;
    int64_t ncoef = 0;        // doubles in the coefficient-gradient array
    int64_t nch = 0;          // 32-sample chunks per channel
    size_t saved_bytes = 0;   // forward activations + checkpoints kept for the backward
    size_t bws_bytes = 0;     // backward workspace
    size_t b_scan = 0, b_part = 0, b_tmp = 0, b_gbuf = 0;  // backward workspace offsets
    int tc_min_taps = tfx::TC_MIN_TAPS;  // FIRs with at least this many taps go to the tensor cores
    bool allow_hiq = true;               // route cascades with poles of radius > 0.999 to FP64 carries
    // device-side coefficient updates (tfx_plan_update_sos): per-section descriptors
    char* dsec = nullptr;  // section descriptors, then FIR descriptors
    int nsec = -1;  // -1: not built yet
    int nfir = 0;
    // the whole chain as one FFT FIR of its composite impulse response
    // (chain_fft); the separate units above stay built for after a
    // coefficient update
    bool use_chain = false;
    int32_t compose_m[16] = {};  // transform size exponent per floor(log2(Lc)) (0: cost model)
    tfx::HostUnit chain;
    int chain_S = 0, chain_L = 0, chain_D = 0;  // sections, combined FIR length, cascade response length
    // trainable chains run by their composite spectrum: the chain unit above
    // (overlap J = chain.L - 1, spectrum from the sections' closed form) runs
    // the forward and, in reverse time, the input gradient
    bool spectral = false;
    tfx::HostUnit spec_fir;  // the FIR (a unit impulse without one) at the chain's transform size
    int spec_nfir = 0;
    int64_t spec_fir_dst = 0;
    size_t off_spec_raw = 0, off_spec_dst = 0;  // every section's raw row and gradient slot, contiguous
    size_t off_spec_z = 0;                      // e^(-2 pi i k / M), k < M (FP64)
    int spec_grid = 0;                          // correlation CTAs
    // the backward's input gradient runs on a side stream (forked from and
    // joined back to the caller's stream by events) while the coefficient
    // gradients' small kernels run on the caller's
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    size_t b_sp_part = 0, b_sp_P = 0, b_sp_w = 0, b_sp_gs = 0;  // backward workspace offsets
};

namespace tfx {
// Tensor-core FIR geometry for NB output blocks per tile (plan.cu).
void tc_geometry(HostUnit& u, int NB);
// Create a plan with a tensor-core tap threshold other than the default.
int plan_create_ex(tfx_plan** out, int64_t C, int64_t N, int64_t ld, const tfx_stage* st, int32_t nst,
                   uint32_t flags, int tc_min_taps, bool allow_hiq = true, const int32_t* compose_m = nullptr);
// Pole radius above which a cascade's cross-tile carries run in FP64.
constexpr double HIQ_RADIUS = 0.999;
// Recompute the plan's section constants on the GPU from raw FP64 rows (design.cu).
int plan_update_sections(tfx_plan* p, const double* rows_dev, cudaStream_t s);
}  // namespace tfx

