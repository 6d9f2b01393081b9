// Fused filter unit: an SOS cascade (chunked parallel scan over time) followed
// by an FIR (sliding window over shared memory), one HBM read of x and one
// HBM write of y per tile.
//
// Operation (TorchFX Sec. 3, lfilter semantics and pipe chaining): per channel,
// each second-order section applies y[n] = b0 x[n] + b1 x[n-1] + b2 x[n-2]
// - a1 y[n-1] - a2 y[n-2] (a0-normalised) with zero initial state, sections in
// order, then y[n] = sum_k h[k] x[n-k].
//
// Decomposition.  A tile is TILE = NTH*T samples of one channel (256 threads x
// 32 samples with an FIR, 128 x 64 without); thread i owns samples
// [i*T, (i+1)*T).  Each section runs as a 2-state recursion with the
// transposed-direct-form-II state W = (w1, w2); over a chunk of T samples the state evolves as
// W_end = A W_start + e, where A = M^T (M the 2x2 one-sample transfer matrix)
// and e is the chunk's zero-state end state.  Per section:
//   1. zero-state pass over the thread's chunk (outputs y_zs, end state e);
//   2. warp Kogge-Stone scan of (A, e) using the powers A^1..A^16, then a
//      Horner combination of the warp totals with A^32;
//   3. decoupled look-back across tiles of the same channel (tile transfer
//      A^NTH) for the tile's incoming state, with bounded waits; each carry
//      and its status travel in one 16-byte word;
//   4. fix-up: y = y_zs + the homogeneous response from the true chunk start
//      state, y_h[t] = -a1 y_h[t-1] - a2 y_h[t-2] (done inside the next
//      section's zero-state pass).
// The FIR then reads the cascade output of this tile plus the last L-1
// cascade outputs of the preceding tile(s), which each tile publishes to
// scratch before the successor needs them (so x == y is safe).
#include "sos_pass.cuh"

namespace tfx {

__device__ __forceinline__ int wphys(int p) { return p + (p >> 5); }

// acc[r] = sum_{k < nkb*R} taps[k] * win[base + r - k], base = FIR_PAD + H + o0.
// Register window xw[m] = win[base_kb - R + m]; taps walked R at a time.
__device__ __forceinline__ void fir_block(const float* __restrict__ win, const float* __restrict__ taps,
                                          int nkb, int base, float (&acc)[FIR_R]) {
    constexpr int R = FIR_R;
    float xw[2 * R];
#pragma unroll
    for (int m = 0; m < 2 * R; ++m) xw[m] = win[wphys(base - R + m)];
    for (int kb = 0; kb < nkb; ++kb) {
        const float4* h4 = reinterpret_cast<const float4*>(taps + kb * R);
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const float4 hv = h4[q];
            const float hk[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kk = 4 * q + j;
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = fmaf(hk[j], xw[R + r - kk], acc[r]);
            }
        }
        const int nb = base - (kb + 1) * R;  // next block's base
#pragma unroll
        for (int m = 2 * R - 1; m >= R; --m) xw[m] = xw[m - R];
#pragma unroll
        for (int m = 0; m < R; ++m) xw[m] = win[wphys(nb - R + m)];
    }
}

// One tile of one unit (the whole CTA).  The tile index comes from the
// caller's ticket, so every predecessor tile of the channel is already running.
template <bool HAS_FIR, int T, int NTH>
__device__ __forceinline__ void unit_tile(const UnitArgs& a, const int64_t tile) {
    constexpr int NW = NTH / 32;
    static_assert(NTH * T == TILE, "tile size");
    extern __shared__ float4 smem_f4[];
    float* smem = reinterpret_cast<float*>(smem_f4);
    __shared__ float2 s_tot[NW];
    __shared__ float2 s_win;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c = tile % a.C;
    const int64_t tt = tile / a.C;
    const int64_t t0 = tt * TILE;
    const int S = a.k.S;

    float u[T];
    load_chunk<T>(a.x + c * a.ldx, t0 + (int64_t)tid * T, a.N, u);

    // Section s's zero-state pass runs fused with the fix-up of section s-1:
    // the fix-up adds the homogeneous response of s-1 from its true chunk start
    // state (yh[t] = -a1 yh[t-1] - a2 yh[t-2]) sample by sample, and the sum is
    // section s's input.
    float2 st = make_float2(0.f, 0.f);  // true chunk start state of the previous section
    float pa1 = 0.f, pa2 = 0.f;         // its feedback coefficients
    for (int s = 0; s <= S; ++s) {
        const bool fix = s > 0, run = s < S;
        float b0 = 0.f, c1 = 0.f, c2 = 0.f, a1 = 0.f, a2 = 0.f;
        if (run) {
            const float* cf = a.k.coef + 8 * s;
            b0 = cf[0]; c1 = cf[1]; c2 = cf[2]; a1 = cf[3]; a2 = cf[4];
        }
        // 1. (fix-up of s-1 +) zero-state pass of s
        float w1, w2;
        section_pass<T>(u, fix, run, b0, c1, c2, a1, a2, st, pa1, pa2, w1, w2);
        if (!run) break;
        const float4* P = a.k.pw + (size_t)s * PW_LEN;

        // 2. warp inclusive scan: v_l = sum_{m<=l} A^m e_{l-m}
        float2 v = make_float2(w1, w2);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float ox = __shfl_up_sync(0xffffffffu, v.x, d);
            const float oy = __shfl_up_sync(0xffffffffu, v.y, d);
            if (lane >= d) {
                const float2 t2 = mv2(P[d], make_float2(ox, oy));
                v.x += t2.x;
                v.y += t2.y;
            }
        }
        if (lane == 31) s_tot[warp] = v;
        const float px = __shfl_up_sync(0xffffffffu, v.x, 1);
        const float py = __shfl_up_sync(0xffffffffu, v.y, 1);
        __syncthreads();

        const float4 A32 = P[32];
        float2 X = make_float2(0.f, 0.f);  // state entering this warp (zero tile-in)
        for (int w = 0; w < warp; ++w) {
            X = mv2(A32, X);
            X.x += s_tot[w].x;
            X.y += s_tot[w].y;
        }
        st = (lane > 0) ? make_float2(px, py) : make_float2(0.f, 0.f);
        {
            const float2 t2 = mv2(P[lane], X);
            st.x += t2.x;
            st.y += t2.y;
        }

        // 3. tile aggregate and decoupled look-back (one thread).  Carries are
        // published and read as single 16-byte words (status travels with the
        // value), so neither side needs a fence.
        if (tid == 0) {
            float2 agg = make_float2(0.f, 0.f);
            for (int w = 0; w < NW; ++w) {
                agg = mv2(A32, agg);
                agg.x += s_tot[w].x;
                agg.y += s_tot[w].y;
            }
            float2 win = make_float2(0.f, 0.f);
            const bool pub = tile != a.drop_tile;
            Carry* mine = a.sc.carry + tile * S + s;
            if (tt == 0) {
                if (pub) publish_carry(mine, 2u, agg);
            } else {
                const float4 AT = P[NTH];
                int64_t j = tile - a.C;
                float2 pv;
                unsigned f = read_carry(a.sc.carry + j * S + s, pv);
                if (f >= 2u) {  // predecessor already inclusive: no aggregate needed
                    win = pv;
                } else {
                    if (pub) publish_carry(mine, 1u, agg);
                    float4 Mp = make_float4(1.f, 0.f, 0.f, 1.f);
                    for (;;) {
                        if (f == 0u) f = wait_carry(a.sc.carry + j * S + s, pv, a.status);
                        if (f == 0u) break;  // gave up: status word records the timeout
                        const float2 t2 = mv2(Mp, pv);
                        win.x += t2.x;
                        win.y += t2.y;
                        if (f >= 2u) break;
                        Mp = mm2(Mp, AT);
                        j -= a.C;
                        f = read_carry(a.sc.carry + j * S + s, pv);
                    }
                }
                float2 incl = mv2(AT, win);
                incl.x += agg.x;
                incl.y += agg.y;
                if (pub) publish_carry(mine, 2u, incl);
            }
            s_win = win;
        }
        __syncthreads();
        {
            const float2 t2 = mv2(P[tid], s_win);
            st.x += t2.x;
            st.y += t2.y;
        }
        pa1 = a1;
        pa2 = a2;
    }

    if constexpr (!HAS_FIR) {
        store_chunk<T>(a.y + c * a.ldy, t0 + (int64_t)tid * T, a.N, u, a.k.gain);
    } else {
        const int H = a.k.H;
        const int nkb = a.k.nkb;
        const int win_len = wphys(FIR_PAD + H + TILE - 1) + 1;
        float* win = smem;
        float* taps = smem + ((win_len + 3) & ~3);

        const int base = FIR_PAD + H + tid * T;
#pragma unroll
        for (int t = 0; t < T; ++t) win[wphys(base + t)] = u[t];
        for (int i = tid; i < FIR_PAD; i += NTH) win[wphys(i)] = 0.f;
        for (int i = tid; i < nkb * FIR_R; i += NTH) taps[i] = a.k.taps[i];
        __syncthreads();

        // publish this tile's last tail_len FIR-input samples for the successor
        const int tl = a.sc.tail_len;
        if (tt + 1 < a.ntt) {
            float* dst = a.sc.tails + tile * (int64_t)tl;
            for (int i = tid; i < tl; i += NTH) dst[i] = win[wphys(FIR_PAD + H + TILE - tl + i)];
            __threadfence();
            __syncthreads();
            if (tid == 0 && tile != a.drop_tile) st_release_u32(a.sc.flags + tile, 1u);
        }

        // halo: samples [t0 - H, t0) at window positions [FIR_PAD, FIR_PAD + H)
        int remaining = H;
        for (int qb = 1; remaining > 0; ++qb) {
            if (tt - qb < 0) {
                for (int i = tid; i < remaining; i += NTH) win[wphys(FIR_PAD + H - ((qb - 1) * TILE + 1 + i))] = 0.f;
                break;
            }
            const int64_t jt = tile - (int64_t)qb * a.C;
            if (tid == 0) wait_flag(a.sc.flags + jt, 1u, a.status);
            __syncthreads();
            const float* src = a.sc.tails + jt * (int64_t)tl;
            const int nq = remaining < tl ? remaining : tl;
            for (int i = tid; i < nq; i += NTH) {
                const int m = (qb - 1) * TILE + 1 + i;  // samples back from t0
                win[wphys(FIR_PAD + H - m)] = __ldcg(src + (tl - 1 - i));
            }
            remaining -= nq;
        }
        __syncthreads();

        float* yrow = a.y + c * a.ldy;
        for (int o0 = tid * FIR_R; o0 < TILE; o0 += NTH * FIR_R) {
            const int64_t n0 = t0 + o0;
            if (n0 >= a.N) break;
            float acc[FIR_R];
#pragma unroll
            for (int r = 0; r < FIR_R; ++r) acc[r] = 0.f;
            fir_block(win, taps, nkb, FIR_PAD + H + o0, acc);
            store_chunk<FIR_R>(yrow, n0, a.N, acc, 1.0f);
        }
    }
}

template <bool HAS_FIR, int T, int NTH>
__global__ void __launch_bounds__(NTH, HAS_FIR ? 2 : 4) k_unit(UnitArgs a) {
    __shared__ unsigned s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(a.sc.ticket, 1u);
    __syncthreads();
    unit_tile<HAS_FIR, T, NTH>(a, s_tile);
}

// Many units (of many clips) in one launch: the ticket runs over the
// concatenated tile ranges of the units (prefix[u] .. prefix[u+1]), so each
// unit's tiles keep their time-major order and look-back stays deadlock-free.
// Buffer pointers in the descriptors are offsets into one of three bases.
template <bool HAS_FIR, int T, int NTH>
__global__ void __launch_bounds__(NTH, HAS_FIR ? 2 : 4)
    k_unit_batched(const BatchUnit* __restrict__ units, const int64_t* __restrict__ prefix, int nunits,
                   unsigned* ticket, BatchBases bases) {
    __shared__ UnitArgs s_args;
    __shared__ int64_t s_tile;
    if (threadIdx.x == 0) {
        const int64_t t = atomicAdd(ticket, 1u);
        int lo = 0, hi = nunits - 1;  // last unit with prefix[u] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchUnit& bu = units[lo];
        UnitArgs a = bu.a;
        a.x = bases.ptr(bu.x_sel) + bu.x_off;
        a.y = bases.ptr(bu.y_sel) + bu.y_off;
        char* w = reinterpret_cast<char*>(bases.ws);
        a.sc.flags = reinterpret_cast<unsigned*>(w + bu.flags_off);
        a.sc.carry = reinterpret_cast<Carry*>(w + bu.carry_off);
        a.sc.tails = reinterpret_cast<float*>(w + bu.tails_off);
        s_args = a;
        s_tile = t - prefix[lo];
    }
    __syncthreads();
    unit_tile<HAS_FIR, T, NTH>(s_args, s_tile);
}

size_t unit_smem_bytes(const UnitConst& k) {
    if (k.L <= 0) return 0;
    const int win_len = (FIR_PAD + k.H + TILE - 1) + ((FIR_PAD + k.H + TILE - 1) >> 5) + 1;
    return (size_t)(((win_len + 3) & ~3) + k.nkb * FIR_R) * sizeof(float);
}

// Raise the kernel's dynamic shared-memory limit once, at plan time, so that
// launches (possibly under stream capture) make no attribute calls.
cudaError_t prepare_unit(const UnitConst& k) {
    static int set_bytes = 48 * 1024;
    const size_t smem = unit_smem_bytes(k);
    if (k.L <= 0 || (int)smem <= set_bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_unit<true, T_CHUNK, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) set_bytes = (int)smem;
    return e;
}

cudaError_t launch_unit_batched(bool has_fir, const BatchUnit* units, const int64_t* prefix, int nunits,
                                int64_t tiles, unsigned* ticket, BatchBases bases, size_t smem, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    if (has_fir)
        k_unit_batched<true, T_CHUNK, NT><<<(unsigned)tiles, NT, smem, s>>>(units, prefix, nunits, ticket, bases);
    else
        k_unit_batched<false, T_CASCADE, NT_CASCADE><<<(unsigned)tiles, NT_CASCADE, 0, s>>>(units, prefix, nunits,
                                                                                           ticket, bases);
    return cudaGetLastError();
}

cudaError_t prepare_unit_batched(size_t smem) {
    static size_t set_bytes = 48 * 1024;
    if (smem <= set_bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_unit_batched<true, T_CHUNK, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) set_bytes = smem;
    return e;
}

cudaError_t launch_unit(const UnitArgs& a, cudaStream_t s) {
    const int64_t tiles = a.C * a.ntt;
    if (tiles <= 0) return cudaSuccess;
    if (a.k.L > 0) {
        k_unit<true, T_CHUNK, NT><<<(unsigned)tiles, NT, unit_smem_bytes(a.k), s>>>(a);
    } else {
        k_unit<false, T_CASCADE, NT_CASCADE><<<(unsigned)tiles, NT_CASCADE, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace tfx
