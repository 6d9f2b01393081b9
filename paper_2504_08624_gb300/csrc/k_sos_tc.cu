// SOS cascade on the tcgen05 tensor cores: chunked state-space form.
//
// Operation (TorchFX Sec. 3, lfilter semantics): per channel, the sections
// in order with zero initial state.  The cascade is one linear system with a
// 2S-dimensional state x (w1, w2 of every section, transposed direct form
// II): x' = A x + B u, y = C x + D u.
//
// Blocks of K = 112 samples.  With s_b the state at the start of block b and
// h the cascade's impulse response,
//     y_b[m]  = sum_{k<=m} h[m-k] u_b[k] + (C A^m) s_b,      m < 112
//     s_(b+1) = A^112 s_b + sum_k (A^(111-k) B) u_b[k].
// GEMM1 (M = 128, N = 128 blocks, K = 112) computes, for every block of a
// tile, the zero-state outputs (rows 0..111: lower-triangular Toeplitz of h)
// and the zero-start end state e_b (rows 112..127: A^(111-k) B).  The scan
// forms the block start states from e (carrying s from tile to tile of the
// segment), and GEMM2 (K = 16) computes the free responses (C A^m) s_b into
// a second accumulator; the epilogue adds the two.
//
// The scan runs eight blocks per step: with Phi = A^112 and the group terms
// G_(g,j) = sum_(i<j) Phi^(j-1-i) e_(8g+i) (Horner: G_1 = e_8g,
// G_(j+1) = Phi G_j + e_(8g+j)), s_(8g+j) = Phi^j s_8g + G_(g,j) for
// j = 1..8, so a tile's 128 blocks take 16 dependent steps; thread
// (j - 1, r) of the 128-thread scan group computes row r of s_(8g+j).
//
// Operands are FP16 hi/lo pairs with three products per K-step (hi*hi,
// hi*lo, lo*hi) and FP32 accumulation in TMEM.  Scales are exact powers of
// two: each constant row is scaled so that its largest entry lies in
// [2^14, 2^15) (the Toeplitz row m and the free-response row m share it),
// each block's samples likewise (tau_b, so a column of the accumulators
// carries its block's scale), and the tile's block start states (rho); the
// epilogue and the scan divide them out.  All operands use the canonical
// no-swizzle K-major layout: element (row, k) at (row % 8) * 16 +
// (row / 8) * SBO + (k % 8) * 2 + (k / 8) * LBO, LBO = 128 bytes and SBO =
// 14 * 128 (K = 112) or 2 * 128 (K = 16).
//
// Persistent kernel, one CTA per SM, 416 threads:
//   warps 0-3    epilogue (TMEM lane quadrant = warp): y = acc1 / (row tau_b) + acc2 / (row rho)
//   warps 4-7    producers: two threads per block (lanes l and l + 16) read its samples in
//                32-byte chunks that do not allocate in L1 -> max -> tau_b -> hi/lo operand
//                stage i % 2; thread 128 prefetches the next tile's samples into L2
//   warps 8-11   scan group; warp 11 (lane quadrant 3) reads the end-state rows
//   warp 12      TMEM allocation; lane 0 issues GEMM1 of tile i, then GEMM2 of tile i - 1
// A CTA walks its segments (g = blockIdx.x + j * gridDim.x) tile by tile;
// every segment starts from zero state.  A segment other than its channel's
// first starts D samples (a whole number of blocks) before its own range and
// discards those outputs: after D samples the true state's free response,
// C A^n s, is below 1e-9 of its initial size (the plan picks D), so the
// state at the segment start is the true one to that accuracy.
// Barriers (all waits bounded, see wait_bar):
//   full[2]      producers -> MMA (operand stage and block scales written)
//   g1_done[2]   GEMM1 committed -> producers (stage free), scan (end states ready)
//   s_ready[2]   scan -> MMA (state operand of tile i written)
//   g2_done[2]   GEMM2 committed -> epilogue (both accumulators ready), scan (state buffer free)
//   acc_free[2]  epilogue -> MMA (accumulator pair drained)
#include "tc_common.cuh"

namespace tfx {
namespace {

constexpr int TCS_THREADS = 416;
constexpr int TCS_PROD = 128;
constexpr int TCS_SCAN0 = 256;  // first scan thread (warp 8)
constexpr int TCS_MMA_WARP = 12;
constexpr int TCS_GROUPS = TCS_NB / 8;             // scan groups of 8 blocks
constexpr uint32_t TCS_SBO1 = (TCS_KB / 8) * 128;  // 1792
constexpr uint32_t TCS_S_BYTES = TCS_NB * 16 * 2;   // one 16-bit [128 blocks x 16] operand
// Row stride of the transposed end states seT[row][block]: a multiple of 4
// (16-byte stores of 4 blocks) that spreads the rows over the banks.
constexpr int TCS_SE_LD = TCS_NB + 4;
constexpr int BAR_PROD = 1, BAR_SCAN = 2;           // named barriers

struct Smem {
    uint8_t a1[2][TCS_A1_BYTES];    // hi, lo
    uint8_t a2[2][TCS_A2_BYTES];    // hi, lo
    uint8_t u[2][2][TCS_A1_BYTES];  // [stage][hi, lo]: [128 blocks x 112]
    uint8_t sop[2][2][TCS_S_BYTES]; // [buffer][hi, lo]: [128 blocks x 16]
    __align__(16) float sf[TCS_NB][16];         // block start states s_b of the tile being scanned
    __align__(16) float seT[16][TCS_SE_LD];     // zero-start block end states, seT[row][b] = e_b[row]
    __align__(16) float sg[TCS_GROUPS][8][16];  // group terms G_(g,j), j = 2..8 at [j - 1]
    __align__(16) float taub[4][TCS_NB];         // 1 / tau_b per tile (ring of 4)
    float rowinv[128];
    uint64_t full[2], g1_done[2], s_ready[2], g2_done[2], acc_free[2];
    float rho[4];  // 1 / rho per tile (ring of 4)
    float red[4];
    uint32_t tmem;
    int ok_prod[2], ok_scan[2];  // shared wait outcomes of the producer and scan groups
};

__device__ __forceinline__ float pow2_scale(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 1.f;
    int sh = 14 - ilogbf(m);
    sh = sh > 126 ? 126 : (sh < -126 ? -126 : sh);
    return ldexpf(1.f, sh);
}

// Iterate the CTA's tiles: segment g = blockIdx.x + j * gridDim.x, tile t of
// the segment, running tile counter i.  The segment's tiles start at s0 (its
// warm-up start) and its outputs are [wlo, whi).
struct TileWalk {
    const SegArgs& a;
    int64_t g, t, i, nt, c, k, s0, wlo, whi;
    __device__ explicit TileWalk(const SegArgs& a_) : a(a_), g(blockIdx.x), t(0), i(0) { load(); }
    __device__ void load() {
        nt = 0;
        if (g >= a.C * a.P) return;
        c = g / a.P;
        k = g % a.P;
        wlo = k * a.Lseg;
        whi = a.N < wlo + a.Lseg ? a.N : wlo + a.Lseg;
        s0 = k > 0 ? wlo - a.D : 0;
        nt = (whi - s0 + TCS_TILE - 1) / TCS_TILE;
    }
    __device__ bool valid() const { return g < a.C * a.P && t < nt; }
    __device__ int64_t n0() const { return s0 + t * TCS_TILE; }
    __device__ void next() {
        ++i;
        if (++t < nt) return;
        t = 0;
        g += gridDim.x;
        load();
        while (g < a.C * a.P && nt == 0) {
            g += gridDim.x;
            load();
        }
    }
};

// dot(row, v) + add for a 16-float row in registers and v in shared memory,
// in four partial sums (v read as four float4).
__device__ __forceinline__ float dot16(const float (&row)[16], const float* v, float add) {
    const float4* v4 = reinterpret_cast<const float4*>(v);
    const float4 q0 = v4[0], q1 = v4[1], q2 = v4[2], q3 = v4[3];
    float p0 = fmaf(row[0], q0.x, add), p1 = row[1] * q0.y, p2 = row[2] * q0.z, p3 = row[3] * q0.w;
    p0 = fmaf(row[4], q1.x, p0);
    p1 = fmaf(row[5], q1.y, p1);
    p2 = fmaf(row[6], q1.z, p2);
    p3 = fmaf(row[7], q1.w, p3);
    p0 = fmaf(row[8], q2.x, p0);
    p1 = fmaf(row[9], q2.y, p1);
    p2 = fmaf(row[10], q2.z, p2);
    p3 = fmaf(row[11], q2.w, p3);
    p0 = fmaf(row[12], q3.x, p0);
    p1 = fmaf(row[13], q3.y, p1);
    p2 = fmaf(row[14], q3.z, p2);
    p3 = fmaf(row[15], q3.w, p3);
    return (p0 + p1) + (p2 + p3);
}

// dot(row, v) + add with v[m] at p[m * ld] (a column of the transposed end states).
__device__ __forceinline__ float dot16_col(const float (&row)[16], const float* p, float add) {
    float p0 = fmaf(row[0], p[0], add), p1 = row[1] * p[TCS_SE_LD], p2 = row[2] * p[2 * TCS_SE_LD],
          p3 = row[3] * p[3 * TCS_SE_LD];
#pragma unroll
    for (int m = 4; m < 16; m += 4) {
        p0 = fmaf(row[m], p[m * TCS_SE_LD], p0);
        p1 = fmaf(row[m + 1], p[(m + 1) * TCS_SE_LD], p1);
        p2 = fmaf(row[m + 2], p[(m + 2) * TCS_SE_LD], p2);
        p3 = fmaf(row[m + 3], p[(m + 3) * TCS_SE_LD], p3);
    }
    return (p0 + p1) + (p2 + p3);
}

__global__ void __launch_bounds__(TCS_THREADS, 1) k_sos_tc(SegArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == TCS_MMA_WARP) {
        tc::tmem_alloc(&sm.tmem, 512u);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(&sm.full[q], TCS_PROD);
            tc::mbar_init(&sm.g1_done[q], 1);
            tc::mbar_init(&sm.s_ready[q], 1);
            tc::mbar_init(&sm.g2_done[q], 1);
            tc::mbar_init(&sm.acc_free[q], 128);
        }
        tc::mbar_init_fence();
    }
    {
        uint4* d1 = reinterpret_cast<uint4*>(&sm.a1[0][0]);
        for (int q = tid; q < 2 * TCS_A1_BYTES / 16; q += TCS_THREADS) d1[q] = a.a1[q];
        uint4* d2 = reinterpret_cast<uint4*>(&sm.a2[0][0]);
        for (int q = tid; q < 2 * TCS_A2_BYTES / 16; q += TCS_THREADS) d2[q] = a.a2[q];
        for (int q = tid; q < 128; q += TCS_THREADS) sm.rowinv[q] = a.rowinv[q];
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = sm.tmem;

    if (warp < 4) {
        // ---------------- epilogue ----------------
        const int m = warp * 32 + lane;  // output phase (TMEM lane)
        const bool act = m < TCS_KB;
        const float rinv = sm.rowinv[m] * a.gain;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (TileWalk w(a); w.valid(); w.next()) {
            const int64_t i = w.i;
            const int q = (int)(i & 1);
            const bool ok = wait_bar(&sm.g2_done[q], (uint32_t)(i >> 1) & 1u, a.status);
            if (!__all_sync(0xffffffffu, ok)) break;  // tcgen05.ld below is warp-collective
            tc::tc_fence_after();
            const float u2 = rinv * sm.rho[i & 3];
            const float* tb = sm.taub[i & 3];
            float* yr = a.y + w.c * a.ldy + w.n0();
            // outputs of the segment's own range only (not its warm-up, not the next segment)
            const int64_t lo = w.wlo - w.n0(), hi = w.whi - w.n0();
            const bool whole = lo <= 0 && hi >= TCS_TILE;
            for (int cc = 0; cc < TCS_NB; cc += 16) {
                float v1[16], v2[16];
                tc::tmem_ld16(tmem + lane_base + (uint32_t)(q * 128 + cc), v1);
                tc::tmem_ld16(tmem + lane_base + (uint32_t)(256 + q * 128 + cc), v2);
                if (act) {
                    float t16[16];  // the 16 blocks' 1 / tau_b, four 16-byte loads
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 t4 = reinterpret_cast<const float4*>(tb + cc)[u];
                        t16[4 * u] = t4.x, t16[4 * u + 1] = t4.y, t16[4 * u + 2] = t4.z, t16[4 * u + 3] = t4.w;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int o = (cc + j) * TCS_KB + m;  // within the tile: 32-bit
                        if (whole || (o >= lo && o < hi)) yr[o] = fmaf(v1[j], rinv * t16[j], v2[j] * u2);
                    }
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&sm.acc_free[q]);
        }
    } else if (warp < 8) {
        // ---------------- producers ----------------
        // lanes l and l + 16 of a producer warp hold the two halves of one block
        // (7 chunks of 8 samples each), so the 8 lanes of a quarter-warp store
        // 8 different blocks' chunks: distinct bank groups of the operand layout
        const int ptid = tid - 128;
        for (TileWalk w(a); w.valid(); w.next()) {
            const int64_t i = w.i;
            const int st = (int)(i & 1);
            if (ptid == 0) {
                // the next tile's samples into L2 while this one is converted: the
                // 16-byte-aligned interior of its range within the channel row
                TileWalk nx = w;
                nx.next();
                if (nx.valid()) {
                    const float* row = a.x + nx.c * a.ldx;
                    const int64_t e = a.N < nx.n0() + TCS_TILE ? a.N : nx.n0() + TCS_TILE;
                    const uintptr_t lo = (reinterpret_cast<uintptr_t>(row + nx.n0()) + 15) & ~uintptr_t(15);
                    const uintptr_t hi = reinterpret_cast<uintptr_t>(row + e) & ~uintptr_t(15);
                    if (hi > lo) tc::bulk_prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
                }
            }
            if (i >= 2) {
                if (ptid == 0) sm.ok_prod[st] = wait_bar(&sm.g1_done[st], (uint32_t)((i - 2) >> 1) & 1u, a.status) ? 1 : 0;
                named_sync(BAR_PROD, TCS_PROD);
                if (!sm.ok_prod[st]) break;
            }
            const float* xr = a.x + w.c * a.ldx;
            const int64_t n0 = w.n0();
            const bool vec = ((reinterpret_cast<uintptr_t>(xr + n0) & 15) == 0);
            const bool vec32 = ((reinterpret_cast<uintptr_t>(xr + n0) & 31) == 0);
            uint8_t* uh = &sm.u[st][0][0];
            uint8_t* ul = &sm.u[st][1][0];
#pragma unroll 1
            for (int it = 0; it < 2; ++it) {
                const int b = it * (TCS_NB / 2) + (ptid >> 5) * 16 + (ptid & 15), half = (ptid >> 4) & 1;
                float v[7][8];
#pragma unroll
                for (int j = 0; j < 7; ++j)
                    load8_32(xr, n0 + (int64_t)b * TCS_KB + 8 * (7 * half + j), a.N, vec32, vec, v[j]);
                float mx = 0.f;
#pragma unroll
                for (int j = 0; j < 7; ++j)
#pragma unroll
                    for (int e = 0; e < 8; ++e) mx = fmaxf(mx, fabsf(v[j][e]));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
                const float tau = pow2_scale(mx);
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    uint4 hi, lo;
                    split8_f16(v[j], tau, hi, lo);
                    const int kc = 7 * half + j;
                    const uint32_t off = (uint32_t)(b >> 3) * TCS_SBO1 + (uint32_t)kc * 128u + (uint32_t)(b & 7) * 16u;
                    *reinterpret_cast<uint4*>(uh + off) = hi;
                    *reinterpret_cast<uint4*>(ul + off) = lo;
                }
                if (half == 0) sm.taub[i & 3][b] = 1.f / tau;
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&sm.full[st]);
        }
    } else if (warp < TCS_MMA_WARP) {
        // ---------------- scan group (warps 8-11) ----------------
        const int sid = tid - TCS_SCAN0;              // 0..127
        const int r = sid & 15, jj = (sid >> 4) + 1;  // chain: row r of s_(8g+jj)
        const int hg = sid >> 3, hr = sid & 7;        // Horner: group hg, rows hr and hr + 8
        const int n2 = 2 * a.S;
        float pj[16], ph0[16], ph1[16];  // Phi^jj row r; Phi rows hr and hr + 8
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            pj[m] = r < n2 ? a.phib[(jj - 1) * 256 + r * 16 + m] : 0.f;
            ph0[m] = hr < n2 ? a.phib[hr * 16 + m] : 0.f;
            ph1[m] = hr + 8 < n2 ? a.phib[(hr + 8) * 16 + m] : 0.f;
        }
        float carry = 0.f;  // threads jj = 8: row r of the tile-out state
        for (TileWalk w(a); w.valid(); w.next()) {
            const int64_t i = w.i;
            const int q = (int)(i & 1);
            if (w.t == 0) carry = 0.f;
            if (sid == 0) {
                bool ok = wait_bar(&sm.g1_done[q], (uint32_t)(i >> 1) & 1u, a.status);
                // the state operand buffer q was read by GEMM2 of tile i - 2
                if (i >= 2) ok = ok && wait_bar(&sm.g2_done[q], (uint32_t)((i - 2) >> 1) & 1u, a.status);
                sm.ok_scan[q] = ok ? 1 : 0;
            }
            named_sync(BAR_SCAN, 128);
            if (!sm.ok_scan[q]) break;
            // end states: warp 11 reads TMEM lanes 96..127 (lanes 16..31: rows 112 + er)
            // and writes row er of seT, four blocks per 16-byte store
            if (warp == 11) {
                tc::tc_fence_after();
                const int er = lane - 16;
                const float einv = er >= 0 ? sm.rowinv[TCS_KB + er] : 0.f;
                const float4* tb4 = reinterpret_cast<const float4*>(sm.taub[i & 3]);
                for (int cc = 0; cc < TCS_NB; cc += 16) {
                    float e[16];
                    tc::tmem_ld16(tmem + (96u << 16) + (uint32_t)(q * 128 + cc), e);
                    if (er >= 0) {
                        float4* dst = reinterpret_cast<float4*>(&sm.seT[er][cc]);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float4 t = tb4[cc / 4 + u];
                            dst[u] = er < n2 ? make_float4(e[4 * u] * einv * t.x, e[4 * u + 1] * einv * t.y,
                                                           e[4 * u + 2] * einv * t.z, e[4 * u + 3] * einv * t.w)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                }
                tc::tc_fence_before();
            }
            if (jj == 8) sm.sf[0][r] = carry;
            named_sync(BAR_SCAN, 128);
            // group terms by Horner, 16 groups in parallel (the 8 threads of a group share a warp):
            // G_2 = Phi e_8g + e_(8g+1) from the end states' column 8g, then G_(j+1) = Phi G_j + e_(8g+j)
            {
                const float* e8 = &sm.seT[0][8 * hg];
                const float g0 = dot16_col(ph0, e8, sm.seT[hr][8 * hg + 1]);
                const float g1 = dot16_col(ph1, e8, sm.seT[hr + 8][8 * hg + 1]);
                sm.sg[hg][1][hr] = g0;
                sm.sg[hg][1][hr + 8] = g1;
                __syncwarp();
                for (int j = 2; j < 8; ++j) {
                    const float* prev = sm.sg[hg][j - 1];
                    const float h0 = dot16(ph0, prev, sm.seT[hr][8 * hg + j]);
                    const float h1 = dot16(ph1, prev, sm.seT[hr + 8][8 * hg + j]);
                    __syncwarp();
                    sm.sg[hg][j][hr] = h0;
                    sm.sg[hg][j][hr + 8] = h1;
                    __syncwarp();
                }
            }
            named_sync(BAR_SCAN, 128);
            // chain: 16 steps of 8 blocks
            for (int g = 0; g < TCS_GROUPS; ++g) {
                const float add = jj == 1 ? sm.seT[r][8 * g] : sm.sg[g][jj - 1][r];
                const float v = r < n2 ? dot16(pj, sm.sf[8 * g], add) : 0.f;
                if (8 * g + jj < TCS_NB) sm.sf[8 * g + jj][r] = v;
                else carry = v;
                named_sync(BAR_SCAN, 128);
            }
            // largest block start state -> rho; the states -> FP16 hi/lo operand
            float smax = 0.f;
            {
                const float4* f4 = reinterpret_cast<const float4*>(&sm.sf[0][0]);
                for (int p = sid; p < TCS_NB * 4; p += 128) {
                    const float4 t = f4[p];
                    smax = fmaxf(fmaxf(smax, fabsf(t.x)), fmaxf(fabsf(t.y), fmaxf(fabsf(t.z), fabsf(t.w))));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
            if (lane == 0) sm.red[warp - 8] = smax;
            named_sync(BAR_SCAN, 128);
            smax = fmaxf(fmaxf(sm.red[0], sm.red[1]), fmaxf(sm.red[2], sm.red[3]));
            const float rho = pow2_scale(smax);
            uint8_t* sh = &sm.sop[q][0][0];
            uint8_t* sl = &sm.sop[q][1][0];
            for (int p = sid; p < TCS_NB * 2; p += 128) {
                const int b = p >> 1, rc = p & 1;
                float v[8];
#pragma unroll
                for (int e2 = 0; e2 < 8; ++e2) v[e2] = sm.sf[b][8 * rc + e2];
                uint4 hi, lo;
                split8_f16(v, rho, hi, lo);
                const uint32_t off = (uint32_t)(b >> 3) * 256u + (uint32_t)rc * 128u + (uint32_t)(b & 7) * 16u;
                *reinterpret_cast<uint4*>(sh + off) = hi;
                *reinterpret_cast<uint4*>(sl + off) = lo;
            }
            tc::fence_proxy_async_smem();
            named_sync(BAR_SCAN, 128);  // also: red and sf are reused by the next tile
            if (sid == 0) {
                sm.rho[i & 3] = 1.f / rho;
                tc::mbar_arrive(&sm.s_ready[q]);
            }
        }
    } else {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16kind_f32(128, TCS_NB, false);
            const uint32_t a1h = tc::smem_u32(&sm.a1[0][0]), a1l = tc::smem_u32(&sm.a1[1][0]);
            const uint32_t a2h = tc::smem_u32(&sm.a2[0][0]), a2l = tc::smem_u32(&sm.a2[1][0]);
            int64_t done2 = 0;  // GEMM2 issued for tiles < done2
            bool alive = true;
            auto gemm2 = [&](int64_t j) -> bool {
                const int q = (int)(j & 1);
                if (!wait_bar(&sm.s_ready[q], (uint32_t)(j >> 1) & 1u, a.status)) return false;
                tc::tc_fence_after();
                const uint32_t sh = tc::smem_u32(&sm.sop[q][0][0]), sl = tc::smem_u32(&sm.sop[q][1][0]);
                const uint32_t d = tmem + (uint32_t)(256 + q * 128);
                const uint64_t dah = tc::desc_noswz(a2h, 128u, 256u), dal = tc::desc_noswz(a2l, 128u, 256u);
                const uint64_t dsh = tc::desc_noswz(sh, 128u, 256u), dsl = tc::desc_noswz(sl, 128u, 256u);
                tc::mma_bf16(d, dah, dsh, idesc, 0u);
                tc::mma_bf16(d, dah, dsl, idesc, 1u);
                tc::mma_bf16(d, dal, dsh, idesc, 1u);
                tc::mma_commit(&sm.g2_done[q]);
                return true;
            };
            for (TileWalk w(a); w.valid(); w.next()) {
                const int64_t i = w.i;
                const int q = (int)(i & 1);
                if (!wait_bar(&sm.full[q], (uint32_t)(i >> 1) & 1u, a.status)) {
                    alive = false;
                    break;
                }
                if (i >= 2 && !wait_bar(&sm.acc_free[q], (uint32_t)((i - 2) >> 1) & 1u, a.status)) {
                    alive = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t uh = tc::smem_u32(&sm.u[q][0][0]), ul = tc::smem_u32(&sm.u[q][1][0]);
                const uint32_t d = tmem + (uint32_t)(q * 128);
                for (int kk = 0; kk < TCS_KB / 16; ++kk) {
                    const uint32_t off = (uint32_t)(2 * kk) * 128u;
                    const uint64_t dah = tc::desc_noswz(a1h + off, 128u, TCS_SBO1);
                    const uint64_t dal = tc::desc_noswz(a1l + off, 128u, TCS_SBO1);
                    const uint64_t dbh = tc::desc_noswz(uh + off, 128u, TCS_SBO1);
                    const uint64_t dbl = tc::desc_noswz(ul + off, 128u, TCS_SBO1);
                    tc::mma_bf16(d, dah, dbh, idesc, kk > 0 ? 1u : 0u);
                    tc::mma_bf16(d, dah, dbl, idesc, 1u);
                    tc::mma_bf16(d, dal, dbh, idesc, 1u);
                }
                tc::mma_commit(&sm.g1_done[q]);
                if (i >= 1) {
                    if (!gemm2(i - 1)) {
                        alive = false;
                        break;
                    }
                    done2 = i;
                }
            }
            // the last tile's GEMM2, then wait for every committed MMA before the TMEM release
            TileWalk last(a);
            int64_t total = 0;
            while (last.valid()) {
                ++total;
                last.next();
            }
            if (alive && total > 0 && done2 == total - 1) {
                if (gemm2(total - 1)) done2 = total;
            }
            if (done2 > 0) wait_bar(&sm.g2_done[(done2 - 1) & 1], (uint32_t)((done2 - 1) >> 1) & 1u, a.status);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == TCS_MMA_WARP) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512u);
    }
}

}  // namespace

size_t sos_tc_smem_bytes() { return sizeof(Smem) + 1024; }

cudaError_t prepare_sos_tc() {
    return cudaFuncSetAttribute(k_sos_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sos_tc_smem_bytes());
}

cudaError_t launch_sos_tc(const SegArgs& a, int grid, cudaStream_t s) {
    if (a.C <= 0 || a.N <= 0) return cudaSuccess;
    const int64_t segs = a.C * a.P;
    const int g = (int)(segs < grid ? segs : grid);
    k_sos_tc<<<(unsigned)g, TCS_THREADS, sos_tc_smem_bytes(), s>>>(a);
    return cudaGetLastError();
}

}  // namespace tfx
