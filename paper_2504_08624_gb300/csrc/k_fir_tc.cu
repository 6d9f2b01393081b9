// Long FIR as a Toeplitz-block GEMM on the tcgen05 tensor cores.
//
// Operation (TorchFX Sec. 3 FIR filters, Table 2 workload): per channel,
// y[n] = sum_{k<L} h[k] x[n-k], causal, zero history.
//
// Formulation.  Outputs are grouped into blocks of P = 128 samples; block n
// needs the input window x[nP - W, nP + P) with W = L - 1 rounded up to 16,
// so with kappa indexing that window,
//     y[nP + i] = sum_kappa A[l][kappa] x[nP - W + kappa],
//     A[l][kappa] = h[i + W - kappa],   i = 127 - l   (TMEM lane l <-> phase i).
// One CTA computes NB output blocks of one channel: D[128 x NB] in TMEM,
// accumulated over K = W + 128 in steps of 16 by tcgen05.mma (M = 128,
// N = NB, K = 16, BF16 operands, FP32 accumulation).
//
// Both operands are Hankel/Toeplitz, and both are expressed with the
// no-swizzle canonical layout without materialising the matrices:
//  * A (taps): A[l][kappa] = g[l + kappa] with g[u] = h[W + 127 - u].  Storing
//    8 copies of g shifted by 0..7 elements, interleaved in 16-byte chunks
//    (chunk j, copy b holds g[8j + b .. 8j + b + 7]), makes every K-step a
//    descriptor with LBO = SBO = 128 bytes starting at chunk 2k.
//  * B (signal): the window is stored in 8-sample chunks, chunk g at column
//    g % 16 and row g / 16 of a [rows x 16] grid laid out column-major
//    (column stride CS = rows * 16 bytes).  Block n's row is then n and the
//    K-step k operand starts at column 2k % 16, row k / 8, with LBO = CS and
//    SBO = 128 bytes.
// FP32-level accuracy from 16-bit products: x = x_hi + x_lo and h = h_hi + h_lo,
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi.  By default the parts are FP16 after
// an exact power-of-two scaling (the tile's window max to [2^14, 2^15), the
// taps likewise), leaving a residual of ~2^-22 of each product; the BF16
// variant leaves ~2^-17, and plain BF16 (hi only) ~2^-9.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace tfx {

// One tile (128 * NB outputs of one channel) on one CTA of 256 threads.
__device__ __forceinline__ void fir_tc_tile(const FirTcArgs& a, const int64_t tile) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int J = a.a_chunks;
    const int rows = a.rows;
    const uint32_t CS = (uint32_t)rows * 16u;
    uint8_t* A_hi = smem;
    uint8_t* A_lo = A_hi + (size_t)J * 128;
    uint8_t* B_hi = A_lo + (size_t)J * 128;
    uint8_t* B_lo = B_hi + (size_t)16 * CS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(B_lo + (size_t)16 * CS);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);

    const int64_t c = tile / a.ntt;
    const int64_t t0 = (tile % a.ntt) * (int64_t)(128 * a.NB);

    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init_fence();
    }

    // taps: both interleaved tables, straight copies
    {
        const uint4* src_hi = a.a_hi;
        const uint4* src_lo = a.a_lo;
        uint4* dhi = reinterpret_cast<uint4*>(A_hi);
        uint4* dlo = reinterpret_cast<uint4*>(A_lo);
        for (int i = tid; i < J * 8; i += blockDim.x) {
            dhi[i] = src_hi[i];
            dlo[i] = src_lo[i];
        }
    }
    // signal window [t0 - W, t0 - W + rows*128) -> hi / lo chunks
    __shared__ float s_red[8];
    const float* xr = a.x + c * a.ldx;
    const int64_t s0 = t0 - a.W;
    const int nchunks = rows * 16;
    const bool vec = ((reinterpret_cast<uintptr_t>(xr + s0) & 15) == 0);
    const bool fp16 = a.mode == FIR_TC_FP16_SPLIT;
    float xscale = 1.f, xunscale = 1.f;
    if (fp16) {
        // per-tile power-of-two scale: window max lands in [2^14, 2^15)
        float m = 0.f;
        for (int g = tid; g < nchunks; g += blockDim.x) {
            float v[8];
            load8(xr, s0 + 8 * (int64_t)g, a.N, vec, v);
#pragma unroll
            for (int i = 0; i < 8; ++i) m = fmaxf(m, fabsf(v[i]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_red[warp] = m;
        __syncthreads();
        m = s_red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_red[w]);
        if (m > 0.f && isfinite(m)) {
            int sh = 14 - ilogbf(m);
            sh = sh > 126 ? 126 : (sh < -126 ? -126 : sh);
            xscale = ldexpf(1.f, sh);
            xunscale = ldexpf(1.f, -sh);
        }
    }
    for (int g = tid; g < nchunks; g += blockDim.x) {
        float v[8];
        load8(xr, s0 + 8 * (int64_t)g, a.N, vec, v);
        uint4 hi, lo;
        if (fp16)
            split8_f16(v, xscale, hi, lo);
        else
            split8_bf16(v, hi, lo);
        const uint32_t off = (uint32_t)(g % 16) * CS + (uint32_t)(g / 16) * 16u;
        *reinterpret_cast<uint4*>(B_hi + off) = hi;
        *reinterpret_cast<uint4*>(B_lo + off) = lo;
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        const uint32_t idesc = tc::idesc_f16kind_f32(128, a.NB, !fp16);
        const uint32_t ahi = tc::smem_u32(A_hi), alo = tc::smem_u32(A_lo);
        const uint32_t bhi = tc::smem_u32(B_hi), blo = tc::smem_u32(B_lo);
        for (int k = 0; k < a.nK; ++k) {
            const uint32_t aoff = (uint32_t)(2 * k) * 128u;
            const uint32_t boff = (uint32_t)((2 * k) & 15) * CS + (uint32_t)(k >> 3) * 16u;
            const uint64_t dah = tc::desc_noswz(ahi + aoff, 128u, 128u);
            const uint64_t dbh = tc::desc_noswz(bhi + boff, CS, 128u);
            tc::mma_bf16(tmem, dah, dbh, idesc, k > 0 ? 1u : 0u);
            if (a.mode != FIR_TC_BF16_PLAIN) {
                const uint64_t dal = tc::desc_noswz(alo + aoff, 128u, 128u);
                const uint64_t dbl = tc::desc_noswz(blo + boff, CS, 128u);
                tc::mma_bf16(tmem, dah, dbl, idesc, 1u);
                tc::mma_bf16(tmem, dal, dbh, idesc, 1u);
            }
        }
        tc::mma_commit(bar);
    }

    // wait for the accumulator (bounded)
    bool ok = true;
    {
        const unsigned long long tw = global_ns();
        while (!tc::mbar_try_wait(bar, 0)) {
            if (global_ns() - tw > WAIT_LIMIT_NS) {
                atomicCAS(a.status, 0, (int)TFX_ERR_TIMEOUT);
                ok = false;
                break;
            }
        }
    }
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
    tc::tc_fence_after();

    if (ok) {
        // epilogue: warp w reads lanes [32 (w%4), +32) and half of the columns
        const int quarter = warp & 3;
        const int nhalf = a.NB / 2;
        const int col0 = (warp >> 2) * nhalf;
        const int l = quarter * 32 + lane;      // TMEM lane = 127 - phase
        const int phase = 127 - l;
        float* yr = a.y + c * a.ldy;
        const float us = a.tap_unscale;
        for (int cc = col0; cc < col0 + nhalf; cc += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cc, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int64_t n = t0 + (int64_t)(cc + j) * 128 + phase;
                if (n < a.N) yr[n] = (v[j] * xunscale) * us;
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

__global__ void __launch_bounds__(256, 1) k_fir_tc(FirTcArgs a) { fir_tc_tile(a, blockIdx.x); }

// FIR tiles of many units (clips) in one launch: block b runs tile
// b - prefix[u] of the unit u with prefix[u] <= b < prefix[u + 1].
__global__ void __launch_bounds__(256, 1)
    k_fir_tc_batched(const BatchFir* __restrict__ units, const int64_t* __restrict__ prefix, int nunits,
                     BatchBases bases) {
    __shared__ FirTcArgs s_args;
    __shared__ int64_t s_tile;
    if (threadIdx.x == 0) {
        const int64_t t = blockIdx.x;
        int lo = 0, hi = nunits - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchFir& bf = units[lo];
        FirTcArgs a = bf.a;
        a.x = bases.ptr(bf.x_sel) + bf.x_off;
        a.y = bases.ptr(bf.y_sel) + bf.y_off;
        s_args = a;
        s_tile = t - prefix[lo];
    }
    __syncthreads();
    fir_tc_tile(s_args, s_tile);
}

cudaError_t launch_fir_tc_batched(const BatchFir* units, const int64_t* prefix, int nunits, int64_t tiles,
                                  BatchBases bases, size_t smem, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    k_fir_tc_batched<<<(unsigned)tiles, 256, smem, s>>>(units, prefix, nunits, bases);
    return cudaGetLastError();
}

cudaError_t prepare_fir_tc_batched(size_t smem) {
    static size_t set_bytes = 48 * 1024;
    if (smem <= set_bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fir_tc_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) set_bytes = smem;
    return e;
}

// ---------------------------------------------------------------------------
// Persistent, warp-specialised variant (one CTA per SM, 416 threads):
//   warps 0-7   producers: signal window of tile i -> hi/lo chunks in stage i%2
//   warps 8-11  epilogue:  accumulator i%2 (TMEM columns 128*(i%2)) -> y
//   warp  12    TMEM allocation; lane 0 issues the MMAs of tile i into
//              accumulator i%2 and commits them to mma_done[i%2]
// The tap tables are loaded once per CTA.  Hand-offs are mbarriers:
//   full[s]      producers -> MMA      (window of stage s written)
//   mma_done[s]  MMA -> producers (stage s free) and epilogue (accumulator s ready)
//   acc_free[s]  epilogue -> MMA       (accumulator s drained)
//   scale_rdy[k] producer -> epilogue  (per-tile FP16 scale, ring of 4)
// Every wait is bounded; on a timeout the status word is set and all roles
// leave their loops, so the CTA always reaches the TMEM release.

namespace {

constexpr int WS_THREADS = 416;
constexpr int WS_PROD = 256;  // producer threads (warps 0-7)
constexpr int WS_MMA_WARP = 12;

}  // namespace

__global__ void __launch_bounds__(WS_THREADS, 1) k_fir_tc_ws(FirTcArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int J = a.a_chunks;
    const int rows = a.rows;
    const uint32_t CS = (uint32_t)rows * 16u;
    const size_t bstage = (size_t)16 * CS;  // bytes of one hi (or lo) window
    uint8_t* A_hi = smem;
    uint8_t* A_lo = A_hi + (size_t)J * 128;
    uint8_t* Bbase = A_lo + (size_t)J * 128;  // [stage][hi, lo]
    uint64_t* bars = reinterpret_cast<uint64_t*>(Bbase + 4 * bstage);
    uint64_t* full = bars;           // [2]
    uint64_t* mma_done = bars + 2;   // [2]
    uint64_t* acc_free = bars + 4;   // [2]
    uint64_t* scale_rdy = bars + 6;  // [4]
    float* s_scale = reinterpret_cast<float*>(bars + 10);  // [4]
    float* s_red = s_scale + 4;                            // [8]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(s_red + 8);
    // producers' shared wait outcome, two slots so that a late reader never
    // sees the next tile's value
    int* s_ok = reinterpret_cast<int*>(tmem_slot + 1);

    if (warp == WS_MMA_WARP) {
        tc::tmem_alloc(tmem_slot, 256u);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(&full[k], WS_PROD);
            tc::mbar_init(&mma_done[k], 1);
            tc::mbar_init(&acc_free[k], 128);  // epilogue threads
        }
        for (int k = 0; k < 4; ++k) tc::mbar_init(&scale_rdy[k], 1);
        tc::mbar_init_fence();
    }
    {
        uint4* dhi = reinterpret_cast<uint4*>(A_hi);
        uint4* dlo = reinterpret_cast<uint4*>(A_lo);
        for (int i = tid; i < J * 8; i += WS_THREADS) {
            dhi[i] = a.a_hi[i];
            dlo[i] = a.a_lo[i];
        }
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t tiles = a.C * a.ntt;
    const int nt = (int)((tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
    const bool fp16 = a.mode == FIR_TC_FP16_SPLIT;

    if (warp < WS_PROD / 32) {
        // ---------------- producers ----------------
        constexpr int U = 4;  // chunks in flight per thread
        const int ptid = tid;
        const int nchunks = rows * 16;
        for (int i = 0; i < nt; ++i) {
            const int st = i & 1;
            if (i >= 2) {
                // one thread waits, a named barrier shares the outcome (uniform exit)
                if (ptid == 0) s_ok[i & 1] = wait_bar(&mma_done[st], ((i - 2) >> 1) & 1, a.status) ? 1 : 0;
                named_sync(2, WS_PROD);
                if (!s_ok[i & 1]) break;
            }
            const int64_t tile = blockIdx.x + (int64_t)i * gridDim.x;
            const int64_t c = tile / a.ntt;
            const int64_t t0 = (tile % a.ntt) * (int64_t)(128 * a.NB);
            const float* xr = a.x + c * a.ldx;
            const int64_t s0 = t0 - a.W;
            const bool vec = ((reinterpret_cast<uintptr_t>(xr + s0) & 15) == 0);
            float xscale = 1.f, xunscale = 1.f;
            if (fp16) {
                float m = 0.f;
                for (int g0 = ptid; g0 < nchunks; g0 += U * WS_PROD) {
                    float v[U][8];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int g = g0 + u * WS_PROD;
                        if (g < nchunks) load8(xr, s0 + 8 * (int64_t)g, a.N, vec, v[u]);
                        else {
#pragma unroll
                            for (int q = 0; q < 8; ++q) v[u][q] = 0.f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int q = 0; q < 8; ++q) m = fmaxf(m, fabsf(v[u][q]));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) s_red[warp] = m;
                named_sync(1, WS_PROD);
                m = s_red[0];
#pragma unroll
                for (int w = 1; w < WS_PROD / 32; ++w) m = fmaxf(m, s_red[w]);
                named_sync(1, WS_PROD);  // s_red is reused by the next tile
                if (m > 0.f && isfinite(m)) {
                    int sh = 14 - ilogbf(m);
                    sh = sh > 126 ? 126 : (sh < -126 ? -126 : sh);
                    xscale = ldexpf(1.f, sh);
                    xunscale = ldexpf(1.f, -sh);
                }
            }
            uint8_t* Bhi = Bbase + (size_t)st * 2 * bstage;
            uint8_t* Blo = Bhi + bstage;
            for (int g0 = ptid; g0 < nchunks; g0 += U * WS_PROD) {
                float v[U][8];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int g = g0 + u * WS_PROD;
                    if (g < nchunks) load8(xr, s0 + 8 * (int64_t)g, a.N, vec, v[u]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int g = g0 + u * WS_PROD;
                    if (g >= nchunks) break;
                    uint4 hi, lo;
                    if (fp16)
                        split8_f16(v[u], xscale, hi, lo);
                    else
                        split8_bf16(v[u], hi, lo);
                    const uint32_t off = (uint32_t)(g % 16) * CS + (uint32_t)(g / 16) * 16u;
                    *reinterpret_cast<uint4*>(Bhi + off) = hi;
                    *reinterpret_cast<uint4*>(Blo + off) = lo;
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&full[st]);
            if (ptid == 0) {
                s_scale[i & 3] = xunscale;
                tc::mbar_arrive(&scale_rdy[i & 3]);
            }
        }
    } else if (warp < WS_MMA_WARP) {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;
        const int l = quarter * 32 + lane;  // TMEM lane = 127 - phase
        const int phase = 127 - l;
        const float us = a.tap_unscale;
        for (int i = 0; i < nt; ++i) {
            const int st = i & 1;
            bool ok = wait_bar(&mma_done[st], (i >> 1) & 1, a.status);
            ok = ok && wait_bar(&scale_rdy[i & 3], (i >> 2) & 1, a.status);
            if (!__all_sync(0xffffffffu, ok)) break;  // tcgen05.ld below is warp-collective
            tc::tc_fence_after();
            const float xu = s_scale[i & 3];
            const int64_t tile = blockIdx.x + (int64_t)i * gridDim.x;
            const int64_t c = tile / a.ntt;
            const int64_t t0 = (tile % a.ntt) * (int64_t)(128 * a.NB);
            float* yr = a.y + c * a.ldy;
            for (int cc = 0; cc < a.NB; cc += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(st * 128 + cc), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int64_t n = t0 + (int64_t)(cc + j) * 128 + phase;
                    if (n < a.N) yr[n] = (v[j] * xu) * us;
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&acc_free[st]);
        }
    } else if (lane == 0) {
        // ---------------- MMA issue ----------------
        const uint32_t idesc = tc::idesc_f16kind_f32(128, a.NB, !fp16);
        const uint32_t ahi = tc::smem_u32(A_hi), alo = tc::smem_u32(A_lo);
        int issued = 0;
        for (int i = 0; i < nt; ++i) {
            const int st = i & 1;
            if (!wait_bar(&full[st], (i >> 1) & 1, a.status)) break;
            if (i >= 2 && !wait_bar(&acc_free[st], ((i - 2) >> 1) & 1, a.status)) break;
            tc::tc_fence_after();
            const uint32_t bhi = tc::smem_u32(Bbase + (size_t)st * 2 * bstage);
            const uint32_t blo = bhi + (uint32_t)bstage;
            const uint32_t d = tmem + (uint32_t)(st * 128);
            for (int k = 0; k < a.nK; ++k) {
                const uint32_t aoff = (uint32_t)(2 * k) * 128u;
                const uint32_t boff = (uint32_t)((2 * k) & 15) * CS + (uint32_t)(k >> 3) * 16u;
                const uint64_t dah = tc::desc_noswz(ahi + aoff, 128u, 128u);
                const uint64_t dbh = tc::desc_noswz(bhi + boff, CS, 128u);
                tc::mma_bf16(d, dah, dbh, idesc, k > 0 ? 1u : 0u);
                if (a.mode != FIR_TC_BF16_PLAIN) {
                    const uint64_t dal = tc::desc_noswz(alo + aoff, 128u, 128u);
                    const uint64_t dbl = tc::desc_noswz(blo + boff, CS, 128u);
                    tc::mma_bf16(d, dah, dbl, idesc, 1u);
                    tc::mma_bf16(d, dal, dbh, idesc, 1u);
                }
            }
            tc::mma_commit(&mma_done[st]);
            issued = i + 1;
        }
        // before the TMEM release: the last committed tile must have completed
        if (issued > 0) wait_bar(&mma_done[(issued - 1) & 1], ((issued - 1) >> 1) & 1, a.status);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == WS_MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 256u);
    }
}

// ---------------------------------------------------------------------------
// Long FIRs (tap tables too large to stay resident): persistent, one CTA per
// SM, 448 threads.  The signal window of a tile stays resident (one buffer:
// a long FIR's MMA time per tile dwarfs the window fill), and the tap tables
// stream through a 2-stage ring in blocks of TC_KBLK K-steps, each block a
// pair of bulk asynchronous copies (hi, lo) issued by a loader warp.
//   warps 0-7   producers: window of tile i (waits for tile i-1's MMAs)
//   warps 8-11  epilogue:  accumulator i%2 -> y
//   warp  12    TMEM allocation; lane 0 issues the MMAs
//   warp  13    lane 0 issues the tap-block copies
// Each tap block accumulates into a fresh TMEM accumulator (the two
// alternate by block), and the epilogue adds the block results into y with
// FP32 round-to-nearest adds: a tensor-core accumulation then spans
// TC_KBLK * 3 * 16 products however long the filter, which keeps the
// accumulation error of 16384-tap FIRs at the level of 1025-tap ones.
// Barriers: b_full (window written), tile_done (tile's MMAs complete: window
// free), acc_ready[2] / acc_free[2] (block accumulators), a_full[2] (tap
// block landed: arrive + transaction bytes), a_empty[2] (tap block
// consumed), scale_rdy[4] (per-tile FP16 scale).

namespace {
constexpr int LG_THREADS = 448;
constexpr int LG_PROD = 256;
constexpr int LG_MMA_WARP = 12;
constexpr int LG_LOAD_WARP = 13;
constexpr int LG_BLOCK_CHUNKS = 2 * TC_KBLK + 16;  // 16-byte-per-copy chunks one tap block spans
}  // namespace

size_t fir_tc_long_smem(int rows) {
    return (size_t)2 * 2 * LG_BLOCK_CHUNKS * 128 + (size_t)2 * 16 * rows * 16 + 16 * 8 + 16 * 4 + 32;
}

__global__ void __launch_bounds__(LG_THREADS, 1) k_fir_tc_long(FirTcArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rows = a.rows;
    const uint32_t CS = (uint32_t)rows * 16u;
    const size_t ablk = (size_t)LG_BLOCK_CHUNKS * 128;  // bytes of one tap block (hi or lo)
    uint8_t* Aring = smem;                              // [stage][hi, lo]
    uint8_t* Bhi = Aring + 4 * ablk;
    uint8_t* Blo = Bhi + (size_t)16 * CS;
    uint64_t* bars = reinterpret_cast<uint64_t*>(Blo + (size_t)16 * CS);
    uint64_t* b_full = bars;         // [1]
    uint64_t* tile_done = bars + 1;  // [1]
    uint64_t* acc_ready = bars + 2;  // [2]
    uint64_t* acc_free = bars + 4;   // [2]
    uint64_t* a_full = bars + 6;     // [2]
    uint64_t* a_empty = bars + 8;    // [2]
    uint64_t* scale_rdy = bars + 10; // [4]
    float* s_scale = reinterpret_cast<float*>(bars + 16);  // [4]
    float* s_red = s_scale + 4;                            // [8]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(s_red + 8);
    int* s_ok = reinterpret_cast<int*>(tmem_slot + 1);  // [2], as in k_fir_tc_ws

    if (warp == LG_MMA_WARP) {
        tc::tmem_alloc(tmem_slot, 256u);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(b_full, LG_PROD);
        tc::mbar_init(tile_done, 1);
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(&acc_ready[k], 1);
            tc::mbar_init(&acc_free[k], 128);
            tc::mbar_init(&a_full[k], 1);
            tc::mbar_init(&a_empty[k], 1);
        }
        for (int k = 0; k < 4; ++k) tc::mbar_init(&scale_rdy[k], 1);
        tc::mbar_init_fence();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t tiles = a.C * a.ntt;
    const int nt = (int)((tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
    const int KB = (a.nK + TC_KBLK - 1) / TC_KBLK;  // tap blocks per tile
    const bool fp16 = a.mode == FIR_TC_FP16_SPLIT;

    if (warp < LG_PROD / 32) {
        // ---------------- producers: the resident window ----------------
        constexpr int U = 4;
        const int ptid = tid;
        const int nchunks = rows * 16;
        for (int i = 0; i < nt; ++i) {
            if (i >= 1) {
                if (ptid == 0) s_ok[i & 1] = wait_bar(tile_done, (i - 1) & 1, a.status) ? 1 : 0;
                named_sync(2, LG_PROD);
                if (!s_ok[i & 1]) break;
            }
            const int64_t tile = blockIdx.x + (int64_t)i * gridDim.x;
            const int64_t c = tile / a.ntt;
            const int64_t t0 = (tile % a.ntt) * (int64_t)(128 * a.NB);
            const float* xr = a.x + c * a.ldx;
            const int64_t s0 = t0 - a.W;
            const bool vec = ((reinterpret_cast<uintptr_t>(xr + s0) & 15) == 0);
            float xscale = 1.f, xunscale = 1.f;
            if (fp16) {
                float m = 0.f;
                for (int g0 = ptid; g0 < nchunks; g0 += U * LG_PROD) {
                    float v[U][8];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int g = g0 + u * LG_PROD;
                        if (g < nchunks) load8(xr, s0 + 8 * (int64_t)g, a.N, vec, v[u]);
                        else {
#pragma unroll
                            for (int q = 0; q < 8; ++q) v[u][q] = 0.f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int q = 0; q < 8; ++q) m = fmaxf(m, fabsf(v[u][q]));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) s_red[warp] = m;
                named_sync(1, LG_PROD);
                m = s_red[0];
#pragma unroll
                for (int w = 1; w < LG_PROD / 32; ++w) m = fmaxf(m, s_red[w]);
                named_sync(1, LG_PROD);
                if (m > 0.f && isfinite(m)) {
                    int sh = 14 - ilogbf(m);
                    sh = sh > 126 ? 126 : (sh < -126 ? -126 : sh);
                    xscale = ldexpf(1.f, sh);
                    xunscale = ldexpf(1.f, -sh);
                }
            }
            for (int g0 = ptid; g0 < nchunks; g0 += U * LG_PROD) {
                float v[U][8];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int g = g0 + u * LG_PROD;
                    if (g < nchunks) load8(xr, s0 + 8 * (int64_t)g, a.N, vec, v[u]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int g = g0 + u * LG_PROD;
                    if (g >= nchunks) break;
                    uint4 hi, lo;
                    if (fp16)
                        split8_f16(v[u], xscale, hi, lo);
                    else
                        split8_bf16(v[u], hi, lo);
                    const uint32_t off = (uint32_t)(g % 16) * CS + (uint32_t)(g / 16) * 16u;
                    *reinterpret_cast<uint4*>(Bhi + off) = hi;
                    *reinterpret_cast<uint4*>(Blo + off) = lo;
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(b_full);
            if (ptid == 0) {
                s_scale[i & 3] = xunscale;
                tc::mbar_arrive(&scale_rdy[i & 3]);
            }
        }
    } else if (warp < LG_MMA_WARP) {
        // ---------------- epilogue: y (+)= block result ----------------
        const int quarter = warp & 3;
        const int l = quarter * 32 + lane;
        const int phase = 127 - l;
        const float us = a.tap_unscale;
        bool alive = true;
        for (int i = 0; i < nt && alive; ++i) {
            bool ok = wait_bar(&scale_rdy[i & 3], (i >> 2) & 1, a.status);
            if (!__all_sync(0xffffffffu, ok)) break;
            const float xu = s_scale[i & 3];
            const int64_t tile = blockIdx.x + (int64_t)i * gridDim.x;
            const int64_t c = tile / a.ntt;
            const int64_t t0 = (tile % a.ntt) * (int64_t)(128 * a.NB);
            float* yr = a.y + c * a.ldy;
            for (int kb = 0; kb < KB; ++kb) {
                const int q = i * KB + kb, acc = q & 1;
                ok = wait_bar(&acc_ready[acc], (q >> 1) & 1, a.status);
                if (!__all_sync(0xffffffffu, ok)) {
                    alive = false;
                    break;
                }
                tc::tc_fence_after();
                for (int cc = 0; cc < a.NB; cc += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * 128 + cc), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int64_t n = t0 + (int64_t)(cc + j) * 128 + phase;
                        if (n < a.N) {
                            const float part = (v[j] * xu) * us;
                            yr[n] = kb == 0 ? part : yr[n] + part;
                        }
                    }
                }
                tc::tc_fence_before();
                tc::mbar_arrive(&acc_free[acc]);
            }
        }
    } else if (warp == LG_MMA_WARP) {
        if (lane == 0) {
            // ---------------- MMA issue ----------------
            const uint32_t idesc = tc::idesc_f16kind_f32(128, a.NB, !fp16);
            const uint32_t bhi = tc::smem_u32(Bhi), blo = tc::smem_u32(Blo);
            int done_tiles = 0;
            bool alive = true;
            for (int i = 0; i < nt && alive; ++i) {
                if (!wait_bar(b_full, i & 1, a.status)) break;
                tc::tc_fence_after();
                for (int kb = 0; kb < KB; ++kb) {
                    const int q = i * KB + kb, st = q & 1, acc = q & 1;
                    if (q >= 2 && !wait_bar(&acc_free[acc], ((q - 2) >> 1) & 1, a.status)) {
                        alive = false;
                        break;
                    }
                    if (!wait_bar(&a_full[st], (q >> 1) & 1, a.status)) {
                        alive = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * 128);
                    const uint32_t ahi = tc::smem_u32(Aring + (size_t)st * 2 * ablk);
                    const uint32_t alo = ahi + (uint32_t)ablk;
                    const int k0 = kb * TC_KBLK;
                    const int k1 = min(a.nK, k0 + TC_KBLK);
                    for (int k = k0; k < k1; ++k) {
                        const uint32_t aoff = (uint32_t)(2 * (k - k0)) * 128u;
                        const uint32_t boff = (uint32_t)((2 * k) & 15) * CS + (uint32_t)(k >> 3) * 16u;
                        const uint64_t dah = tc::desc_noswz(ahi + aoff, 128u, 128u);
                        const uint64_t dbh = tc::desc_noswz(bhi + boff, CS, 128u);
                        tc::mma_bf16(d, dah, dbh, idesc, k > k0 ? 1u : 0u);  // fresh per block
                        if (a.mode != FIR_TC_BF16_PLAIN) {
                            const uint64_t dal = tc::desc_noswz(alo + aoff, 128u, 128u);
                            const uint64_t dbl = tc::desc_noswz(blo + boff, CS, 128u);
                            tc::mma_bf16(d, dah, dbl, idesc, 1u);
                            tc::mma_bf16(d, dal, dbh, idesc, 1u);
                        }
                    }
                    tc::mma_commit(&a_empty[st]);
                    tc::mma_commit(&acc_ready[acc]);
                }
                if (!alive) break;
                tc::mma_commit(tile_done);
                done_tiles = i + 1;
            }
            if (done_tiles > 0) wait_bar(tile_done, (done_tiles - 1) & 1, a.status);
        }
    } else if (warp == LG_LOAD_WARP && lane == 0) {
        // ---------------- tap-block loader ----------------
        const int total = nt * KB;
        int issued = 0;
        for (int q = 0; q < total; ++q) {
            const int st = q & 1, kb = q % KB;
            if (q >= 2 && !wait_bar(&a_empty[st], ((q - 2) >> 1) & 1, a.status)) break;
            const int k0 = kb * TC_KBLK;
            const int k1 = min(a.nK, k0 + TC_KBLK);
            const uint32_t bytes = (uint32_t)(2 * (k1 - 1 - k0) + 18) * 128u;
            uint8_t* dst = Aring + (size_t)st * 2 * ablk;
            tc::mbar_arrive_expect_tx(&a_full[st], 2u * bytes);
            tc::bulk_g2s(dst, a.a_hi + (size_t)(2 * k0) * 8, bytes, &a_full[st]);
            tc::bulk_g2s(dst + ablk, a.a_lo + (size_t)(2 * k0) * 8, bytes, &a_full[st]);
            issued = q + 1;
        }
        // copies still in flight must land before the CTA exits
        for (int q = issued - 2 < 0 ? 0 : issued - 2; q < issued; ++q)
            wait_bar(&a_full[q & 1], (q >> 1) & 1, a.status);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == LG_MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 256u);
    }
}

size_t fir_tc_smem_bytes(const FirTcArgs& a) {
    if (a.persistent == 2) return fir_tc_long_smem(a.rows);
    if (a.persistent == 1)
        return (size_t)a.a_chunks * 128 * 2 + (size_t)16 * a.rows * 16 * 4 + 10 * 8 + 12 * 4 + 32;
    return (size_t)a.a_chunks * 128 * 2 + (size_t)16 * a.rows * 16 * 2 + 16;
}

cudaError_t prepare_fir_tc(size_t smem) {
    static size_t set_bytes = 0;
    cudaError_t e = cudaSuccess;
    if (smem > set_bytes) {
        e = cudaFuncSetAttribute(k_fir_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) set_bytes = smem;
    }
    return e;
}

cudaError_t prepare_fir_tc_ws(size_t smem) {
    static size_t set_bytes = 0;
    if (smem <= set_bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fir_tc_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) set_bytes = smem;
    return e;
}

cudaError_t prepare_fir_tc_long(size_t smem) {
    static size_t set_bytes = 0;
    if (smem <= set_bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fir_tc_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) set_bytes = smem;
    return e;
}

cudaError_t launch_fir_tc(const FirTcArgs& a, cudaStream_t s) {
    const int64_t tiles = a.C * a.ntt;
    if (tiles <= 0) return cudaSuccess;
    const int64_t grid = tiles < a.grid ? tiles : a.grid;
    if (a.persistent == 2) {
        k_fir_tc_long<<<(unsigned)grid, LG_THREADS, fir_tc_smem_bytes(a), s>>>(a);
    } else if (a.persistent == 1) {
        k_fir_tc_ws<<<(unsigned)grid, WS_THREADS, fir_tc_smem_bytes(a), s>>>(a);
    } else {
        k_fir_tc<<<(unsigned)tiles, 256, fir_tc_smem_bytes(a), s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace tfx
