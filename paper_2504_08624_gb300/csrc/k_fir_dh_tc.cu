// FIR tap gradient on the tcgen05 tensor cores.
//
// For an FIR stage with input u and output gradient g (the filters as network
// layers, TorchFX Sec. 3):  dL/dh_k = sum_c sum_n g[c][n] u[c][n - k].
//
// Formulation.  Cut every channel into blocks of 128 samples and number the
// blocks of all channels r = c R + r' (R = ceil(N / 128)).  With n = 128 r' + j,
//     X[j][q] = sum_r A[j][r] B[q][r],   A[j][r] = g[c][128 r' + j],
//                                        B[q][r] = u[c][128 r' + 127 - q - k0],
//     dL/dh_{k0 + q + j - 127} = sum over j of X[j][q]   (anti-diagonal sums),
// for the lag window [k0, k0 + LW); q runs over NQ = LW + 127 rounded up to
// 16.  So the correlation is one GEMM with M = 128 phases, N = NQ shifted
// copies of the input and K = all blocks of all channels, followed by a
// diagonal reduction of its 128 x NQ result.
//
// One CTA per (K range, lag window); 416 threads:
//   warps 0-7   producers: stage each K-step's raw FP32 data (16 blocks of g
//               and the u samples its B rows span, both contiguous) into a
//               5-slot shared ring with cp.async four K-steps ahead, then
//               gather A (128 x 16) and B (NQ x 16) from it, split each value
//               into BF16 hi + lo, and store both in the canonical K-major
//               no-swizzle layout of a 3-stage operand ring; K-steps at
//               channel ends or signal edges read global memory directly.
//               They also write the time-reversed g, which the FIR's
//               input-gradient pass consumes, when asked to
//   warps 8-11  epilogue: after the last K-step, each thread reads its TMEM
//               lane j (one row of X), 16 columns at a time, into a shared
//               tile; one thread per lag then sums that lag's anti-diagonal
//               (fixed order: bit-reproducible), and the CTA writes its
//               partial dh
//   warp 12     allocates TMEM; lane 0 issues A_hi B_hi + A_hi B_lo + A_lo B_hi
//               (M = 128, N <= 256 per instruction, K = 16, FP32 accumulation
//               over the whole K range)
// Every wait is bounded; on a timeout the status word is set and all roles
// leave their loops, so the CTA always reaches the TMEM release.
#include "tc_common.cuh"

namespace tfx {
namespace {

constexpr int DT_THREADS = 416;
constexpr int DT_PROD = 256;
constexpr int DT_MMA_WARP = 12;
constexpr int DT_STAGES = 3;
constexpr int DT_LW_MAX = 385;  // one window covers up to this many lags (NQ <= 512)
constexpr int DT_DH_WORDS = 512;
constexpr uint32_t DT_A_BYTES = 2 * 128 * 16;  // one part (hi or lo) of A: 2 K-chunks x 128 rows x 16 B

__host__ __device__ inline uint32_t dt_b_bytes(int NQ) { return 2u * (uint32_t)NQ * 16u; }
__host__ __device__ inline uint32_t dt_stage_bytes(int NQ) { return 2 * DT_A_BYTES + 2 * dt_b_bytes(NQ); }
// one raw staging slot: 2048 samples of g and 2048 + NQ - 128 of u, FP32
__host__ __device__ inline uint32_t dt_raw_bytes(int NQ) { return (uint32_t)(2048 + 2048 + NQ - 128) * 4u; }

constexpr int DT_RAW = 5;  // raw staging slots: four K-steps ahead

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct ChunkMap {
    bool valid, isA;
    int row, kc;
    uint32_t off;
};

// Split 8 FP32 values into BF16 hi + lo, two at a time with the paired conversions.
__device__ __forceinline__ void split8_bf16x2(const float (&v)[8], uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
        h[i] = *reinterpret_cast<const uint32_t*>(&hb);
        l[i] = *reinterpret_cast<const uint32_t*>(&lb);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

}  // namespace

__global__ void __launch_bounds__(DT_THREADS, 1)
    k_fir_dh_tc(const float* __restrict__ g, int64_t ldg, int g_rev, const float* __restrict__ u, int64_t ldu,
                float* __restrict__ gflip, int64_t C, int64_t N, int64_t R, int64_t nks, int L, int LW, int NQ,
                float* __restrict__ part, int* status) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t STAGE = dt_stage_bytes(NQ);
    const uint32_t BB = dt_b_bytes(NQ);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)DT_STAGES * STAGE + (size_t)DT_RAW * dt_raw_bytes(NQ));
    uint64_t* full = bars;              // [DT_STAGES <= 4] producers -> MMA
    uint64_t* empty = bars + 4;         // [DT_STAGES <= 4] MMA -> producers
    uint64_t* done = bars + 8;          // [1] MMA -> epilogue
    float* dh_s = reinterpret_cast<float*>(bars + 9);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dh_s + DT_DH_WORDS);
    int* s_ok = reinterpret_cast<int*>(tmem_slot + 1);  // [2]

    const int64_t k0 = (int64_t)blockIdx.y * LW;
    const int lw = (int)min((int64_t)LW, (int64_t)L - k0);
    const int G = gridDim.x;
    const int64_t ks0 = (int64_t)blockIdx.x * nks / G;
    const int nk = (int)((int64_t)(blockIdx.x + 1) * nks / G - ks0);
    const uint32_t ncols = NQ <= 128 ? 128u : (NQ <= 256 ? 256u : 512u);
    const int64_t nblk = C * R;

    if (warp == DT_MMA_WARP) {
        tc::tmem_alloc(tmem_slot, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < DT_STAGES; ++k) {
            tc::mbar_init(&full[k], DT_PROD);
            tc::mbar_init(&empty[k], 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_init_fence();
    }
    for (int i = tid; i < DT_DH_WORDS; i += DT_THREADS) dh_s[i] = 0.f;
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < DT_PROD / 32) {
        // ---------------- producers ----------------
        float* const gf = blockIdx.y == 0 ? gflip : nullptr;  // one lag window writes it
        const int nA = 256, nch = 256 + 2 * NQ;
        // this thread's chunks (the same in every K-step): A rows j / B rows q,
        // K-chunk kc, and the 16-byte slot in the stage
        constexpr int U = 4;
        constexpr int MAXC = (256 + 2 * 512 + DT_PROD - 1) / DT_PROD;  // chunks per thread, at most
        ChunkMap maps[2 * U];
#pragma unroll
        for (int k = 0; k < 2 * U; ++k) {
            const int it = k / U, uu = k % U;
            const int ch = tid + it * U * DT_PROD + uu * DT_PROD;
            ChunkMap cm;
            cm.valid = ch < nch;
            cm.isA = ch < nA;
            cm.row = cm.isA ? (ch & 127) : ((ch - nA) % NQ);
            cm.kc = cm.isA ? (ch >> 7) : ((ch - nA) / NQ);
            cm.off = (uint32_t)cm.kc * (cm.isA ? 128u * 16u : (uint32_t)NQ * 16u) + (uint32_t)cm.row * 16u;
            maps[k] = cm;
        }
        static_assert(MAXC <= 2 * U, "chunk map too small");
        // raw FP32 staging ring, DT_RAW - 1 K-steps ahead (cp.async)
        static_assert(DT_STAGES <= 4, "barrier slots");
        const int BRAW = 2048 + NQ - 128;  // u samples one K-step's B rows span
        const int RAWF = 2048 + BRAW;
        float* raw = reinterpret_cast<float*>(smem + (size_t)DT_STAGES * STAGE);
        const bool base_al = ((reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(u)) & 15) == 0;
        // (channel, block) cursors advanced 16 blocks per K-step (no division in
        // the loop): one for the K-step being converted, one for the prefetch
        struct Cursor {
            int64_t c, rq;
        };
        auto advance = [&](Cursor& cu, int64_t nb) {
            cu.rq += nb;
            while (cu.rq >= R) {
                cu.rq -= R;
                ++cu.c;
            }
        };
        Cursor cur{(ks0 * 16) / R, (ks0 * 16) % R};
        Cursor pfc = cur;
        // A K-step is staged when its 16 blocks lie in one channel and both raw
        // ranges (2048 samples of g, BRAW of u) are inside the signal and
        // 16-byte aligned; other K-steps (channel ends, signal edges) load directly.
        auto staged = [&](int64_t rb, const Cursor& cu, int64_t& aoff, int64_t& boff) -> bool {
            if (!base_al || rb + 16 > nblk) return false;
            const int64_t a0 = 128 * cu.rq, m0 = a0 + 128 - NQ - k0;
            if (cu.rq + 16 > R || a0 + 2048 > N || m0 < 0 || m0 + BRAW > N) return false;
            aoff = g_rev ? cu.c * ldg + (N - 2048 - a0) : cu.c * ldg + a0;
            boff = cu.c * ldu + m0;
            return ((aoff | boff) & 3) == 0;
        };
        auto prefetch = [&](int i) {
            int64_t aoff, boff;
            if (i < nk && staged((ks0 + i) * 16, pfc, aoff, boff)) {
                float* dst = raw + (size_t)(i % DT_RAW) * RAWF;
                for (int q = tid; q < 512; q += DT_PROD) cp_async16(dst + 4 * q, g + aoff + 4 * q);
                for (int q = tid; q < BRAW / 4; q += DT_PROD) cp_async16(dst + 2048 + 4 * q, u + boff + 4 * q);
            }
            cp_async_commit();  // one group per K-step, empty or not
            advance(pfc, 16);
        };
        for (int i = 0; i < DT_RAW - 1; ++i) prefetch(i);
        for (int i = 0; i < nk; ++i, advance(cur, 16)) {
            const int st = i % DT_STAGES;
            // everyone is done with K-step i-1 (whose raw slot the prefetch below
            // refills) and, once the ring is full, the MMA has released stage st;
            // one thread waits and a named barrier shares the outcome (two slots,
            // so a late reader never sees the next iteration's value)
            if (tid == 0)
                s_ok[i & 1] = (i < DT_STAGES || wait_bar(&empty[st], ((i - DT_STAGES) / DT_STAGES) & 1, status)) ? 1 : 0;
            named_sync(1, DT_PROD);
            if (!s_ok[i & 1]) break;
            prefetch(i + DT_RAW - 1);
            cp_async_wait<DT_RAW - 1>();  // this thread's copies for K-step i have landed
            named_sync(1, DT_PROD);      // and everyone else's
            const int64_t rb0 = (ks0 + i) * 16;  // first block of this K-step
            int64_t aoff_i, boff_i;
            const bool stg = staged(rb0, cur, aoff_i, boff_i);
            const float* rawA = raw + (size_t)(i % DT_RAW) * RAWF;
            const float* rawB = rawA + 2048;
            uint8_t* Ah = smem + (size_t)st * STAGE;
            uint8_t* Al = Ah + DT_A_BYTES;
            uint8_t* Bh = Al + DT_A_BYTES;
            uint8_t* Bl = Bh + BB;
            // (channel, block) of the first block of each K-chunk of 8 blocks, and
            // whether all 8 blocks lie in that channel
            const int64_t cb0 = cur.c, rq0 = cur.rq;
            Cursor c8 = cur;
            advance(c8, 8);
            const int64_t cb1 = c8.c, rq1 = c8.rq;
            const bool one0 = rb0 + 8 <= nblk && rq0 + 8 <= R;
            const bool one1 = rb0 + 16 <= nblk && rq1 + 8 <= R;
#pragma unroll
            for (int it = 0; it < 2; ++it) {  // at most 1280 chunks: two passes of U x 256
                const int ch0 = tid + it * U * DT_PROD;
                if (ch0 >= nch) break;
                float v[U][8];
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    const ChunkMap cm = maps[it * U + uu];
                    if (!cm.valid) continue;
                    const int kc = cm.kc;
                    if (stg) {  // from the staged raw data
                        if (cm.isA) {
                            if (g_rev) {
#pragma unroll
                                for (int e = 0; e < 8; ++e) v[uu][e] = rawA[2047 - 128 * (8 * kc + e) - cm.row];
                            } else {
#pragma unroll
                                for (int e = 0; e < 8; ++e) v[uu][e] = rawA[128 * (8 * kc + e) + cm.row];
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 8; ++e) v[uu][e] = rawB[128 * (8 * kc + e) + NQ - 1 - cm.row];
                        }
                        continue;
                    }
                    const int64_t c0 = kc ? cb1 : cb0, r0 = kc ? rq1 : rq0;
                    const bool onek = kc ? one1 : one0;
                    if (cm.isA) {
                        const int64_t n0 = 128 * r0 + cm.row;  // sample of the first block
                        const float* gr = g + c0 * ldg;
                        if (onek && n0 + 128 * 7 < N) {
                            if (g_rev) {
#pragma unroll
                                for (int e = 0; e < 8; ++e) v[uu][e] = gr[N - 1 - (n0 + 128 * e)];
                            } else {
#pragma unroll
                                for (int e = 0; e < 8; ++e) v[uu][e] = gr[n0 + 128 * e];
                            }
                            continue;
                        }
                    } else {
                        const int64_t m0 = 128 * r0 + 127 - cm.row - k0;
                        if (onek && m0 >= 0 && m0 + 128 * 7 < N) {
                            const float* ur = u + c0 * ldu + m0;
#pragma unroll
                            for (int e = 0; e < 8; ++e) v[uu][e] = ur[128 * e];
                            continue;
                        }
                    }
                    // general case: blocks crossing a channel end or the signal edges
                    int64_t c = c0, rp = r0;
                    const int64_t rb = rb0 + 8 * kc;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        float val = 0.f;
                        if (rb + e < nblk) {
                            if (cm.isA) {
                                const int64_t n = 128 * rp + cm.row;
                                if (n < N) val = g_rev ? g[c * ldg + (N - 1 - n)] : g[c * ldg + n];
                            } else {
                                const int64_t m = 128 * rp + 127 - cm.row - k0;
                                if (m >= 0 && m < N) val = u[c * ldu + m];
                            }
                        }
                        v[uu][e] = val;
                        if (++rp == R) {
                            rp = 0;
                            ++c;
                        }
                    }
                }
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    const ChunkMap cm = maps[it * U + uu];
                    if (!cm.valid) break;
                    uint4 hi, lo;
                    split8_bf16x2(v[uu], hi, lo);
                    *reinterpret_cast<uint4*>((cm.isA ? Ah : Bh) + cm.off) = hi;
                    *reinterpret_cast<uint4*>((cm.isA ? Al : Bl) + cm.off) = lo;
                    if (cm.isA && gf && stg) {  // the reversed gradient, for the FIR's input-gradient pass
                        float* gb = gf + cur.c * N + (N - 1 - 128 * cur.rq - cm.row - 1024 * cm.kc);
#pragma unroll
                        for (int e = 0; e < 8; ++e) gb[-128 * e] = v[uu][e];
                    } else if (cm.isA && gf) {
                        const int kc = cm.kc;
                        int64_t c = kc ? cb1 : cb0, rp = kc ? rq1 : rq0;
                        const int64_t rb = rb0 + 8 * kc;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int64_t n = 128 * rp + cm.row;
                            if (rb + e < nblk && n < N) gf[c * N + (N - 1 - n)] = v[uu][e];
                            if (++rp == R) {
                                rp = 0;
                                ++c;
                            }
                        }
                    }
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&full[st]);
        }
        cp_async_wait<0>();  // no copy left in flight
    } else if (warp < DT_MMA_WARP) {
        // ---------------- epilogue ----------------
        // X is read 16 columns at a time into a shared tile (the stage ring is
        // idle once `done` fired); each lag's anti-diagonal is then summed by one
        // thread in a fixed order, so the result is bit-reproducible
        const int et = tid - DT_PROD;  // 0..127
        const bool ok = nk > 0 && wait_bar(done, 0, status);
        const bool all_ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
        float* tile = reinterpret_cast<float*>(smem);  // [128][17]
        if (all_ok) tc::tc_fence_after();
        const int quarter = warp & 3;
        const int j = quarter * 32 + lane;  // TMEM lane = row of X = phase j
        for (int q0 = 0; q0 < NQ; q0 += 16) {
            float v[16];
            if (all_ok) {
                tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)q0, v);
            } else {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) v[jj] = 0.f;
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) tile[j * 17 + jj] = v[jj];
            named_sync(2, 128);
            // lags fed by columns [q0, q0 + 16): k = q + j - 127 in [q0 - 127, q0 + 15]
            for (int k = q0 - 127 + et; k <= q0 + 15; k += 128) {
                if (k < 0 || k >= lw) continue;
                float acc = 0.f;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int jr = k + 127 - (q0 + jj);
                    if (jr >= 0 && jr < 128) acc += tile[jr * 17 + jj];
                }
                dh_s[k] += acc;
            }
            named_sync(2, 128);
        }
        for (int i = tid - DT_PROD; i < lw; i += 128) part[(k0 + i) * G + blockIdx.x] = dh_s[i];
    } else if (lane == 0) {
        // ---------------- MMA issue ----------------
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int st = i % DT_STAGES;
            if (!wait_bar(&full[st], (i / DT_STAGES) & 1, status)) break;
            tc::tc_fence_after();
            const uint32_t ah = tc::smem_u32(smem + (size_t)st * STAGE);
            const uint32_t al = ah + DT_A_BYTES;
            const uint32_t bh = al + DT_A_BYTES;
            const uint32_t bl = bh + BB;
            const uint64_t dah = tc::desc_noswz(ah, 128u * 16u, 128u);
            const uint64_t dal = tc::desc_noswz(al, 128u * 16u, 128u);
            for (int n0 = 0; n0 < NQ; n0 += 256) {
                const int nc = NQ - n0 < 256 ? NQ - n0 : 256;
                const uint32_t idesc = tc::idesc_f16kind_f32(128, nc, true);
                const uint64_t dbh = tc::desc_noswz(bh + (uint32_t)n0 * 16u, (uint32_t)NQ * 16u, 128u);
                const uint64_t dbl = tc::desc_noswz(bl + (uint32_t)n0 * 16u, (uint32_t)NQ * 16u, 128u);
                const uint32_t d = tmem + (uint32_t)n0;
                tc::mma_bf16(d, dah, dbh, idesc, i > 0 ? 1u : 0u);
                tc::mma_bf16(d, dah, dbl, idesc, 1u);
                tc::mma_bf16(d, dal, dbh, idesc, 1u);
            }
            tc::mma_commit(&empty[st]);
            issued = i + 1;
        }
        if (issued == nk) {
            tc::mma_commit(done);
        }
        // before the TMEM release: the last committed K-step must have completed
        if (issued > 0) wait_bar(&empty[(issued - 1) % DT_STAGES], ((issued - 1) / DT_STAGES) & 1, status);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == DT_MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, ncols);
    }
}

// Geometry of the tap-gradient GEMM: lag windows of LW (NQ rows of B each)
// and G K-range CTAs per window (every CTA gets at least one K-step).
void fir_dh_tc_geometry(int64_t C, int64_t N, int L, int sm_count, int* G, int* nwin, int* LW, int* NQ) {
    const int lw = L <= DT_LW_MAX ? L : 384;
    *LW = lw;
    *NQ = (lw + 127 + 15) / 16 * 16;
    *nwin = (L + lw - 1) / lw;
    const int64_t R = (N + 127) / 128;
    const int64_t nks = (C * R + 15) / 16;
    int64_t g = sm_count / *nwin;
    if (g < 1) g = 1;
    if (g > nks) g = nks;
    if (g < 1) g = 1;
    *G = (int)g;
}

// At least 120 KB, so that one CTA (and its up to 512 TMEM columns) holds an SM.
size_t fir_dh_tc_smem(int NQ) {
    const size_t need = (size_t)DT_STAGES * dt_stage_bytes(NQ) + (size_t)DT_RAW * dt_raw_bytes(NQ) + 9 * sizeof(uint64_t) +
                        DT_DH_WORDS * sizeof(float) + 16;
    return need > 120 * 1024 ? need : 120 * 1024;
}

cudaError_t prepare_fir_dh_tc() {
    return cudaFuncSetAttribute(k_fir_dh_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fir_dh_tc_smem(512));
}

cudaError_t launch_fir_dh_tc(const float* g, int64_t ldg, int g_rev, const float* u, int64_t ldu, float* gflip,
                             int64_t C, int64_t N, int L, int sm_count, float* part, int* status, cudaStream_t s) {
    if (C <= 0 || N <= 0) return cudaSuccess;
    int G, nwin, LW, NQ;
    fir_dh_tc_geometry(C, N, L, sm_count, &G, &nwin, &LW, &NQ);
    const int64_t R = (N + 127) / 128;
    const int64_t nks = (C * R + 15) / 16;
    dim3 grid((unsigned)G, (unsigned)nwin);
    k_fir_dh_tc<<<grid, DT_THREADS, fir_dh_tc_smem(NQ), s>>>(g, ldg, g_rev, u, ldu, gflip, C, N, R, nks, L, LW, NQ,
                                                              part, status);
    return cudaGetLastError();
}

}  // namespace tfx
