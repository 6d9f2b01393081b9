// Backward (adjoint) kernels: gradients of a filter chain with respect to its
// input signal and its coefficients, for the filters used as differentiable
// layers (TorchFX Sec. 3: the filters are torch modules inside a network).
//
// SOS section, a0-normalised: y = (B/A) u.  For L = sum g*y with g = dL/dy:
//   lambda  = (1/A)^T g        lambda[n] = g[n] - a1 lambda[n+1] - a2 lambda[n+2]
//   dL/du   = (B/A)^T g        the section run backwards in time over g
//   dL/db_k =  sum_n lambda[n] u[n-k]   (k = 0, 1, 2)
//   dL/da_k = -sum_n lambda[n] y[n-k]   (k = 1, 2)
// FIR with taps h: dL/du = h correlated with g (the FIR over g reversed in
// time), dL/dh_k = sum_n g[n] u[n-k].
//
// k_sos_bwd runs a whole cascade's adjoint in reverse time on the warp-tile
// geometry of the training forward (32 lanes x 32 samples per tile):
//   1. each lane recomputes every section's output over its chunk from the
//      chunk-start states the forward stored (block-boundary checkpoints),
//      keeping the upper half of them in shared memory; when the reverse
//      sweep reaches the lower half, those are recomputed into the freed
//      slots (S/2 + 1 slots instead of S + 1, for occupancy);
//   2. per section, last to first: a zero-state reverse pass over the chunk
//      gives lambda and dL/du with zero state beyond the chunk; the chunk
//      states (lambda[n0], lambda[n0+1]) are combined by a reverse
//      Kogge-Stone shuffle scan and a decoupled look-back over the later
//      tiles of the channel, with the transposed powers of the forward chunk
//      transfer matrix (the adjoint one-sample transfer is the transpose of
//      the forward one); the homogeneous fix-up from the true incoming state
//      then completes lambda, the section's dL/du (whose state is a linear
//      map of the incoming lambda state, so no numerator cancels), and the
//      chunk's coefficient partial sums, in the same loop as the next
//      section's zero-state pass.
// Coefficient partials are summed per tile in FP32 and across tiles in FP64.
#include "tfx_common.cuh"

namespace tfx {

constexpr int BWD_WPB = 2;  // warps (tiles) per CTA
constexpr unsigned FULL = 0xffffffffu;

// m^T v for a row-major 2x2 matrix m = (m00 m01 m10 m11)
__device__ __forceinline__ float2 mv2t(float4 m, float2 v) {
    return make_float2(fmaf(m.x, v.x, m.z * v.y), fmaf(m.y, v.x, m.w * v.y));
}

// v[i] = sample n0 + i of a row (zero beyond N); rev: sample n sits at row[N-1-n]
template <int T>
__device__ __forceinline__ void bwd_load(const float* row, int64_t n0, int64_t N, bool rev, float (&v)[T]) {
    if (!rev) {
        const float* p = row + n0;
        if (n0 + T <= N && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
            const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
            for (int q = 0; q < T / 4; ++q) {
                const float4 w = p4[q];
                v[4 * q] = w.x;
                v[4 * q + 1] = w.y;
                v[4 * q + 2] = w.z;
                v[4 * q + 3] = w.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < T; ++i) v[i] = (n0 + i < N) ? p[i] : 0.f;
        }
    } else {
        const int64_t base = N - n0 - T;  // where sample n0 + T - 1 sits
        if (base >= 0 && ((reinterpret_cast<uintptr_t>(row + base) & 15) == 0)) {
            const float4* p4 = reinterpret_cast<const float4*>(row + base);
#pragma unroll
            for (int q = 0; q < T / 4; ++q) {
                const float4 w = p4[q];
                v[T - 1 - 4 * q] = w.x;
                v[T - 2 - 4 * q] = w.y;
                v[T - 3 - 4 * q] = w.z;
                v[T - 4 - 4 * q] = w.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < T; ++i) v[i] = (n0 + i < N) ? row[N - 1 - (n0 + i)] : 0.f;
        }
    }
}

template <int T>
__device__ __forceinline__ void bwd_store(float* row, int64_t n0, int64_t N, bool rev, const float (&v)[T]) {
    if (!rev) {
        float* p = row + n0;
        if (n0 + T <= N && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
            float4* p4 = reinterpret_cast<float4*>(p);
#pragma unroll
            for (int q = 0; q < T / 4; ++q) p4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < T; ++i)
                if (n0 + i < N) p[i] = v[i];
        }
    } else {
        const int64_t base = N - n0 - T;
        if (base >= 0 && ((reinterpret_cast<uintptr_t>(row + base) & 15) == 0)) {
            float4* p4 = reinterpret_cast<float4*>(row + base);
#pragma unroll
            for (int q = 0; q < T / 4; ++q)
                p4[q] = make_float4(v[T - 1 - 4 * q], v[T - 2 - 4 * q], v[T - 3 - 4 * q], v[T - 4 - 4 * q]);
        } else {
#pragma unroll
            for (int i = 0; i < T; ++i)
                if (n0 + i < N) row[N - 1 - (n0 + i)] = v[i];
        }
    }
}

// Coefficients of the section being fixed up, with its true incoming adjoint
// state p = (lambda[n0+T], lambda[n0+T+1]).
struct FixSec {
    float a1, a2, c1, c2, d;
    float2 p;
};
struct RunSec {
    float b0, c1, c2, a1, a2;
};
struct Partials {
    float db0, db1, db2, da1, da2;
};

// One reverse pass over a lane's chunk.  FIX: complete lambda and dL/du of the
// fixed section (gr holds its zero-state dL/du, lam its zero-state lambda),
// accumulating the coefficient partials against its input xi and output xo.
// RUN: zero-state pass of the next section over the resulting gradient.
// Returns the zero-state chunk state (lambda_zs[0], lambda_zs[1]).
template <int T, bool FIX, bool RUN>
__device__ __forceinline__ float2 bwd_pass(float (&gr)[T], float (&lam)[T], const float* xi, const float* xo,
                                           const FixSec& f, const RunSec& r, Partials& pt) {
    float h1 = f.p.x, h2 = f.p.y, l1 = f.p.x, l2 = f.p.y;
    float s1 = 0.f, s2 = 0.f;
    if (FIX) {
        s1 = fmaf(f.c1, f.p.x, f.c2 * f.p.y);
        s2 = fmaf(f.c2, f.p.x, f.d * f.p.y);
    }
    float y1 = 0.f, y2 = 0.f;
    float q1 = 0.f, q2 = 0.f, w1 = 0.f, w2 = 0.f;
#pragma unroll
    for (int t = T - 1; t >= 0; --t) {
        float v = gr[t];
        if (FIX) {
            const float h = fmaf(-f.a1, h1, -f.a2 * h2);
            h2 = h1;
            h1 = h;
            const float l = lam[t] + h;
            const float ui = xi[t * 32], uo = xo[t * 32];
            pt.db0 = fmaf(ui, l, pt.db0);
            pt.db1 = fmaf(ui, l1, pt.db1);
            pt.db2 = fmaf(ui, l2, pt.db2);
            pt.da1 = fmaf(uo, l1, pt.da1);
            pt.da2 = fmaf(uo, l2, pt.da2);
            l2 = l1;
            l1 = l;
            float yh;
            if (t == T - 1) yh = s1;
            else if (t == T - 2) yh = fmaf(-f.a1, y1, s2);
            else yh = fmaf(-f.a1, y1, -f.a2 * y2);
            y2 = y1;
            y1 = yh;
            v += yh;
        }
        if (RUN) {
            const float l = fmaf(-r.a1, q1, fmaf(-r.a2, q2, v));
            q2 = q1;
            q1 = l;
            lam[t] = l;
            gr[t] = fmaf(r.b0, v, w1);
            const float n1 = fmaf(r.c1, v, fmaf(-r.a1, w1, w2));
            w2 = fmaf(r.c2, v, -r.a2 * w1);
            w1 = n1;
        } else {
            gr[t] = v;
        }
    }
    return make_float2(q1, q2);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Shared-memory slots per warp for the section outputs u_0 (cascade input) ..
// u_S.  Only u_{S1} .. u_S (S1 = S / 2) are kept at first; once the upper
// sections are done, u_0 .. u_{S1-1} are recomputed into the freed slots.
__host__ __device__ constexpr int bwd_slots(int S) {
    return (S - S / 2 + 1) > (S / 2 + 1) ? (S - S / 2 + 1) : (S / 2 + 1);
}

template <int T>
__global__ void __launch_bounds__(32 * BWD_WPB, 8) k_sos_bwd(BwdArgs a) {
    extern __shared__ float4 bwd_smem4[];
    const int lane = threadIdx.x & 31;
    const int S = a.k.S;
    const int S1 = S / 2;
    const int NS = bwd_slots(S);
    // per-warp slots [NS][T][32 lanes]: upper phase u_k in slot k - S1 (k >= S1);
    // lower phase u_k in slot k + 1 (k < S1), u_{S1} staying in slot 0
    float* stk = reinterpret_cast<float*>(bwd_smem4) + (size_t)(threadIdx.x >> 5) * NS * T * 32 + lane;

    unsigned tk = 0;
    if (lane == 0) tk = atomicAdd(a.ticket, 1u);
    tk = __shfl_sync(FULL, tk, 0);
    const int64_t tiles = a.C * a.ntt;
    if ((int64_t)tk >= tiles) return;  // the grid is rounded up to whole CTAs
    const int64_t c = (int64_t)tk % a.C;
    const int64_t rt = (int64_t)tk / a.C;  // reverse time-tile index: 0 = the channel's last tile
    const int64_t tt = a.ntt - 1 - rt;
    const int64_t chunk = tt * 32 + lane;
    const int64_t n0 = chunk * T;

    // 1. recompute the section outputs of this chunk from the stored chunk-start
    //    states, keeping u_{S1} .. u_S
    {
        float r[T];
        bwd_load<T>(a.u0 + c * a.ldu, n0, a.N, false, r);
        if (S1 == 0) {
#pragma unroll
            for (int t = 0; t < T; ++t) stk[t * 32] = r[t];
        }
        for (int s = 0; s < S; ++s) {
            float2 st = make_float2(0.f, 0.f);
            if (chunk < a.nch) st = a.ckpt[(c * S + s) * a.nch + chunk];
            const float* cf = a.k.coef + 8 * s;
            const float b0 = cf[0], c1 = cf[1], c2 = cf[2], a1 = cf[3], a2 = cf[4];
            float w1 = st.x, w2 = st.y;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float v = r[t];
                r[t] = fmaf(b0, v, w1);
                const float n1 = fmaf(c1, v, fmaf(-a1, w1, w2));
                w2 = fmaf(c2, v, -a2 * w1);
                w1 = n1;
            }
            if (s + 1 >= S1) {
                float* o = stk + (size_t)(s + 1 - S1) * T * 32;
#pragma unroll
                for (int t = 0; t < T; ++t) o[t * 32] = r[t];
            }
        }
    }

    // 2. sections last to first, in reverse time
    float gr[T], lam[T];
    bwd_load<T>(a.g + c * a.ldg, n0, a.N, a.g_rev != 0, gr);
#pragma unroll
    for (int t = 0; t < T; ++t) lam[t] = 0.f;
    FixSec f{0.f, 0.f, 0.f, 0.f, 0.f, make_float2(0.f, 0.f)};
    for (int it = 0; it <= S; ++it) {
        const int sf = S - it;      // section fixed up in this pass (if < S)
        const int sr = S - 1 - it;  // section whose zero-state pass runs (if >= 0)
        RunSec r{0.f, 0.f, 0.f, 0.f, 0.f};
        if (sr >= 0) {
            const float* cf = a.k.coef + 8 * sr;
            r = RunSec{cf[0], cf[1], cf[2], cf[3], cf[4]};
        }
        if (sf == S1 - 1) {
            // lower phase: u_0 .. u_{S1-1} into slots 1 .. S1 (the upper sections'
            // slots are free now), streaming through shared memory
            float* d0 = stk + (size_t)T * 32;
            const float* row = a.u0 + c * a.ldu;
            if (n0 + T <= a.N && ((reinterpret_cast<uintptr_t>(row + n0) & 15) == 0)) {
                const float4* p4 = reinterpret_cast<const float4*>(row + n0);
#pragma unroll
                for (int q = 0; q < T / 4; ++q) {
                    const float4 w = p4[q];
                    d0[(4 * q) * 32] = w.x;
                    d0[(4 * q + 1) * 32] = w.y;
                    d0[(4 * q + 2) * 32] = w.z;
                    d0[(4 * q + 3) * 32] = w.w;
                }
            } else {
#pragma unroll
                for (int t = 0; t < T; ++t) d0[t * 32] = (n0 + t < a.N) ? row[n0 + t] : 0.f;
            }
            for (int k = 1; k < S1; ++k) {
                float2 st0 = make_float2(0.f, 0.f);
                if (chunk < a.nch) st0 = a.ckpt[(c * S + (k - 1)) * a.nch + chunk];
                const float* cf = a.k.coef + 8 * (k - 1);
                const float b0 = cf[0], c1 = cf[1], c2 = cf[2], a1 = cf[3], a2 = cf[4];
                const float* src = stk + (size_t)k * T * 32;
                float* dst = stk + (size_t)(k + 1) * T * 32;
                float w1 = st0.x, w2 = st0.y;
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float v = src[t * 32];
                    dst[t * 32] = fmaf(b0, v, w1);
                    const float n1 = fmaf(c1, v, fmaf(-a1, w1, w2));
                    w2 = fmaf(c2, v, -a2 * w1);
                    w1 = n1;
                }
            }
        }
        // slots holding the fixed section's input u_sf and output u_{sf+1}
        const int sfx = sf < S ? sf : S1;
        const float* xi = stk + (size_t)(sfx >= S1 ? sfx - S1 : sfx + 1) * T * 32;
        const float* xo = stk + (size_t)(sfx + 1 >= S1 ? (sfx + 1 == S1 ? 0 : sfx + 1 - S1) : sfx + 2) * T * 32;
        Partials pt{0.f, 0.f, 0.f, 0.f, 0.f};
        float2 e;
        if (it == 0) e = bwd_pass<T, false, true>(gr, lam, xi, xo, f, r, pt);
        else if (sr >= 0) e = bwd_pass<T, true, true>(gr, lam, xi, xo, f, r, pt);
        else e = bwd_pass<T, true, false>(gr, lam, xi, xo, f, r, pt);
        if (sf < S) {
            pt.db0 = warp_sum(pt.db0);
            pt.db1 = warp_sum(pt.db1);
            pt.db2 = warp_sum(pt.db2);
            pt.da1 = warp_sum(pt.da1);
            pt.da2 = warp_sum(pt.da2);
            if (lane == 0) {  // column-major partials: [S * 5][tiles]
                float* pp = a.part + (int64_t)(sf * 5) * tiles + tk;
                pp[0] = pt.db0;
                pp[tiles] = pt.db1;
                pp[2 * tiles] = pt.db2;
                pp[3 * tiles] = -pt.da1;
                pp[4 * tiles] = -pt.da2;
            }
        }
        if (sr < 0) break;

        // 3. reverse scan of the chunk states: v_l = sum_{m >= l} At^(m-l) e_m,
        //    At = transpose of the forward chunk transfer A
        const float4* P = a.k.pw + (size_t)sr * PW_LEN;
        float2 v = e;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float4 Pd = P[d];
            const float ox = __shfl_down_sync(FULL, v.x, d);
            const float oy = __shfl_down_sync(FULL, v.y, d);
            if (lane + d < 32) {
                const float2 t2 = mv2t(Pd, make_float2(ox, oy));
                v.x += t2.x;
                v.y += t2.y;
            }
        }
        const float nx = __shfl_down_sync(FULL, v.x, 1);
        const float ny = __shfl_down_sync(FULL, v.y, 1);
        const float ax = __shfl_sync(FULL, v.x, 0);
        const float ay = __shfl_sync(FULL, v.y, 0);

        // 4. decoupled look-back over the later tiles of the channel (lane L
        //    probes the tile L+1 steps later): win = sum_m At32^m v_(rt-1-m)
        float2 win = make_float2(0.f, 0.f);
        {
            const float2 agg = make_float2(ax, ay);
            Carry* mine = a.carry + (int64_t)tk * S + sr;
            if (rt == 0) {
                if (lane == 0) publish_carry(mine, 2u, agg);
            } else {
                const float4 PL = P[32 * lane];
                float4 Mw = make_float4(1.f, 0.f, 0.f, 1.f);
                int64_t jr0 = rt - 1;
                bool published = false;
                for (;;) {
                    const int64_t jr = jr0 - lane;
                    float2 pv = make_float2(0.f, 0.f);
                    unsigned fl = 2u;  // past the channel's end: zero, inclusive
                    if (jr >= 0) fl = read_carry(a.carry + (jr * a.C + c) * S + sr, pv);
                    const unsigned incl_mask = __ballot_sync(FULL, fl >= 2u);
                    const unsigned none_mask = __ballot_sync(FULL, fl == 0u);
                    if (!published && !(incl_mask & 1u)) {
                        if (lane == 0) publish_carry(mine, 1u, agg);
                        published = true;
                    }
                    const int first = incl_mask ? (__ffs(incl_mask) - 1) : 32;
                    const unsigned need = first >= 31 ? FULL : ((2u << first) - 1u);
                    if (none_mask & need) {
                        const int wl = __ffs(none_mask & need) - 1;
                        unsigned got = 1u;
                        if (lane == wl) {
                            float2 dummy;
                            got = wait_carry(a.carry + (jr * a.C + c) * S + sr, dummy, a.status);
                        }
                        got = __shfl_sync(FULL, got, wl);
                        if (got == 0u) break;  // gave up: the status word records the timeout
                        continue;
                    }
                    float2 cntb = make_float2(0.f, 0.f);
                    if (lane <= first) cntb = mv2t(mm2(Mw, PL), pv);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        cntb.x += __shfl_xor_sync(FULL, cntb.x, o);
                        cntb.y += __shfl_xor_sync(FULL, cntb.y, o);
                    }
                    win.x += cntb.x;
                    win.y += cntb.y;
                    if (first < 32) break;
                    Mw = mm2(Mw, P[1024]);
                    jr0 -= 32;
                }
                if (lane == 0) {
                    float2 incl = mv2t(P[32], win);
                    incl.x += agg.x;
                    incl.y += agg.y;
                    publish_carry(mine, 2u, incl);
                }
            }
        }
        // true incoming adjoint state of this lane's chunk for section sr
        float2 p = lane < 31 ? make_float2(nx, ny) : make_float2(0.f, 0.f);
        const float2 t2 = mv2t(P[31 - lane], win);
        p.x += t2.x;
        p.y += t2.y;
        f = FixSec{r.a1, r.a2, r.c1, r.c2, a.k.coef[8 * sr + 5], p};
    }
    if (a.gout) bwd_store<T>(a.gout + c * a.ldo, n0, a.N, a.out_rev != 0, gr);
}

size_t sos_bwd_smem_bytes(int S) { return (size_t)BWD_WPB * bwd_slots(S) * T_CHUNK * 32 * sizeof(float); }

cudaError_t prepare_sos_bwd(int S) {
    if (S < 1 || S > BWD_SMAX) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_sos_bwd<T_CHUNK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sos_bwd_smem_bytes(BWD_SMAX));
}

cudaError_t launch_sos_bwd(const BwdArgs& a, cudaStream_t s) {
    const int64_t tiles = a.C * a.ntt;
    if (tiles <= 0) return cudaSuccess;
    if (a.k.S < 1 || a.k.S > BWD_SMAX) return cudaErrorInvalidValue;
    const int64_t ctas = (tiles + BWD_WPB - 1) / BWD_WPB;
    k_sos_bwd<T_CHUNK><<<(unsigned)ctas, 32 * BWD_WPB, sos_bwd_smem_bytes(a.k.S), s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// time reversal of rows: y[c][n] = x[c][N-1-n]

__global__ void k_flip_rows(const float* __restrict__ x, float* __restrict__ y, int64_t C, int64_t N, int64_t ldx,
                            int64_t ldy, int vec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = blockIdx.y; c < C; c += gridDim.y) {
        const float* xr = x + c * ldx;
        float* yr = y + c * ldy;
        if (vec) {  // N, ldx, ldy multiples of 4 and 16-byte aligned rows
            const int64_t n4 = N / 4;
            const float4* x4 = reinterpret_cast<const float4*>(xr);
            float4* y4 = reinterpret_cast<float4*>(yr);
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
                const float4 v = x4[n4 - 1 - i];
                y4[i] = make_float4(v.w, v.z, v.y, v.x);
            }
        } else {
            for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += stride)
                yr[n] = xr[N - 1 - n];
        }
    }
}

cudaError_t launch_flip_rows(const float* x, float* y, int64_t C, int64_t N, int64_t ldx, int64_t ldy,
                             cudaStream_t s) {
    if (C <= 0 || N <= 0) return cudaSuccess;
    const int vec = (N % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(y) & 15) == 0)
                        ? 1
                        : 0;
    const int bs = 256;
    const int64_t per_row = vec ? N / 4 : N;
    int64_t gx = (per_row + bs - 1) / bs;
    if (gx > 1024) gx = 1024;
    const int64_t gy = C < 65535 ? C : 65535;
    k_flip_rows<<<dim3((unsigned)gx, (unsigned)gy), bs, 0, s>>>(x, y, C, N, ldx, ldy, vec);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FIR tap gradient on CUDA cores (plans that keep FIRs off the tensor cores):
// part[k][blk] = sum over the DH_BLOCK samples n of block blk of g[n] u[n-k],
// k < L.  One warp per block,
// lane l owns samples [64 l, 64 l + 64) of it; lags are walked in windows of
// DH_WIN staged in shared memory, 16 lags per register pass.  Shared arrays
// are padded by one word per 64 (index i at i + i/64) so that the 32 lanes'
// 64-sample strides fall in distinct banks.

constexpr int DH_WPB = 2;
constexpr int DH_SEG = DH_BLOCK / 32;  // samples per lane
static_assert(DH_SEG == 64, "the padding scheme assumes 64 samples per lane");
__device__ __forceinline__ int dh_phys(int i) { return i + (i >> 6); }
constexpr int DH_G_WORDS = DH_BLOCK + DH_BLOCK / 64;
constexpr int DH_U_LEN = DH_BLOCK + DH_WIN;
constexpr int DH_U_WORDS = DH_U_LEN + DH_U_LEN / 64 + 1;

int64_t fir_dh_rows(int64_t C, int64_t N) { return C * ((N + DH_BLOCK - 1) / DH_BLOCK); }

__global__ void __launch_bounds__(32 * DH_WPB) k_fir_dh(const float* __restrict__ g, int64_t ldg, int g_rev,
                                                        const float* __restrict__ u, int64_t ldu, int64_t C,
                                                        int64_t N, int64_t nbpc, int L, int Lp,
                                                        float* __restrict__ part) {
    __shared__ float sg_all[DH_WPB][DH_G_WORDS];
    __shared__ float su_all[DH_WPB][DH_U_WORDS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t blk = (int64_t)blockIdx.x * DH_WPB + w;
    if (blk >= C * nbpc) return;  // whole warp leaves together
    float* sg = sg_all[w];
    float* su = su_all[w];
    const int64_t c = blk / nbpc;
    const int64_t nb0 = (blk % nbpc) * DH_BLOCK;
    const float* grow = g + c * ldg;
    const float* urow = u + c * ldu;
    for (int i = lane; i < DH_BLOCK; i += 32) {
        const int64_t n = nb0 + i;
        float v = 0.f;
        if (n < N) v = g_rev ? grow[N - 1 - n] : grow[n];
        sg[dh_phys(i)] = v;
    }
    const int nwin = (L + DH_WIN - 1) / DH_WIN;
    for (int wi = 0; wi < nwin; ++wi) {
        __syncwarp();
        // su[i] holds u[mbase + i], mbase = nb0 - DH_WIN (wi + 1)
        const int64_t mbase = nb0 - (int64_t)DH_WIN * (wi + 1);
        for (int i = lane; i < DH_U_LEN; i += 32) {
            const int64_t m = mbase + i;
            su[dh_phys(i)] = (m >= 0 && m < N) ? urow[m] : 0.f;
        }
        __syncwarp();
        const int kbn = min(DH_WIN / 16, (L - wi * DH_WIN + 15) / 16);
        for (int kb = 0; kb < kbn; ++kb) {
            // acc[r] = sum_j g[64 lane + j] u[64 lane + j - (wi DH_WIN + 16 kb + r)]
            // su index of that u: 64 lane + j - 16 kb - r + DH_WIN
            float acc[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) acc[r] = 0.f;
            const int ub = DH_SEG * lane + DH_WIN - 16 * kb - 16;  // xw[m] = su[ub + 16 jb + m]
            float xw[32];  // at block jb: xw[m] = su[ub + 16 jb + m]
#pragma unroll
            for (int m = 16; m < 32; ++m) xw[m] = su[dh_phys(ub + m - 16)];
#pragma unroll
            for (int jb = 0; jb < DH_SEG / 16; ++jb) {
#pragma unroll
                for (int m = 0; m < 16; ++m) xw[m] = xw[m + 16];
#pragma unroll
                for (int m = 16; m < 32; ++m) xw[m] = su[dh_phys(ub + 16 * jb + m)];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const float gv = sg[dh_phys(DH_SEG * lane + 16 * jb + jj)];
#pragma unroll
                    for (int r = 0; r < 16; ++r) acc[r] = fmaf(gv, xw[jj - r + 16], acc[r]);
                }
            }
            // reduce-scatter of the 16 sums over the warp: lane 2r ends with lag r
#pragma unroll
            for (int o = 16, n = 8; o >= 2; o >>= 1, n >>= 1) {
                const bool up = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < n; ++i) {
                    const float send = up ? acc[i] : acc[i + n];
                    const float recv = __shfl_xor_sync(FULL, send, o);
                    acc[i] = (up ? acc[i + n] : acc[i]) + recv;
                }
            }
            acc[0] += __shfl_xor_sync(FULL, acc[0], 1);
            const int k = wi * DH_WIN + 16 * kb + (lane >> 1);
            if ((lane & 1) == 0 && k < L) part[(int64_t)k * (C * nbpc) + blk] = acc[0];  // [L][blocks]
        }
    }
}

cudaError_t launch_fir_dh(const float* g, int64_t ldg, int g_rev, const float* u, int64_t ldu, int64_t C,
                          int64_t N, int L, int Lp, float* part, cudaStream_t s) {
    if (C <= 0 || N <= 0) return cudaSuccess;
    if (L < 1 || Lp < L || (Lp & 15) != 0) return cudaErrorInvalidValue;
    const int64_t nbpc = (N + DH_BLOCK - 1) / DH_BLOCK;
    const int64_t blocks = C * nbpc;
    k_fir_dh<<<(unsigned)((blocks + DH_WPB - 1) / DH_WPB), 32 * DH_WPB, 0, s>>>(g, ldg, g_rev, u, ldu, C, N,
                                                                              nbpc, L, Lp, part);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 column sums of column-major FP32 partials: out[col] = sum_r part[col][r].
// One CTA per column; the rows are read contiguously and reduced in a tree.

__global__ void k_colsum(const float* __restrict__ part, int64_t rows, double* __restrict__ out) {
    __shared__ double red[8];
    const float* p = part + (int64_t)blockIdx.x * rows;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) acc += (double)p[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        out[blockIdx.x] = s;
    }
}

cudaError_t launch_colsum(const float* part, int64_t rows, int ncol, double* out, cudaStream_t s) {
    if (ncol <= 0) return cudaSuccess;
    k_colsum<<<(unsigned)ncol, 256, 0, s>>>(part, rows, out);
    return cudaGetLastError();
}

// Section gradients from the normalised-coefficient sums (sums[s*5 + 0..4]:
// b0 b1 b2 a1 a2) to the raw row (b0 b1 b2 a0 a1 a2), whose normalised values
// are b/a0 and a/a0:
//   dL/db_k = G_bk / a0,  dL/da_k = G_ak / a0 (k = 1, 2),
//   dL/da0  = -(sum_k (b_k/a0) G_bk + sum_k (a_k/a0) G_ak) / a0.
__global__ void k_sos_grad_finalize(const double* __restrict__ sums, int S, const double* __restrict__ raw,
                                    const int64_t* __restrict__ dst, double* __restrict__ dcoef) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double* G = sums + 5 * s;
    const double* r = raw + 6 * s;
    const double inv = 1.0 / r[3];
    double* o = dcoef + dst[s];
    o[0] = G[0] * inv;
    o[1] = G[1] * inv;
    o[2] = G[2] * inv;
    o[4] = G[3] * inv;
    o[5] = G[4] * inv;
    o[3] = -(r[0] * G[0] + r[1] * G[1] + r[2] * G[2] + r[4] * G[3] + r[5] * G[4]) * inv * inv;
}

cudaError_t launch_sos_grad_finalize(const double* sums, int S, const double* raw, const int64_t* dst,
                                     double* dcoef, cudaStream_t s) {
    if (S <= 0) return cudaSuccess;
    k_sos_grad_finalize<<<(unsigned)((S + 63) / 64), 64, 0, s>>>(sums, S, raw, dst, dcoef);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Mean squared error and its gradient: loss = mean((y - t)^2),
// g = 2 (y - t) / (C N).  The loss is accumulated in FP64 (one atomic per CTA).

__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ g, int64_t C,
                      int64_t N, int64_t ld, double inv, double* __restrict__ loss, int flat4) {
    __shared__ double red[8];
    const float ginv = (float)(2.0 * inv);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // per-thread sums in FP32 (a few dozen terms each; FP64 arithmetic is slow
    // on this part), combined in FP64 across threads and CTAs
    float accf = 0.f;
    if (flat4) {  // dense rows (ld == N), 16-byte aligned, C N a multiple of 4
        const int64_t n4 = C * N / 4;
        const float4* y4 = reinterpret_cast<const float4*>(y);
        const float4* t4 = reinterpret_cast<const float4*>(t);
        float4* g4 = reinterpret_cast<float4*>(g);
        for (int64_t i = i0; i < n4; i += stride) {
            const float4 a = y4[i], b = t4[i];
            const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
            if (g) g4[i] = make_float4(d0 * ginv, d1 * ginv, d2 * ginv, d3 * ginv);
            accf = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, accf))));
        }
    } else {
        for (int64_t c = 0; c < C; ++c) {
            const int64_t o = c * ld;
            for (int64_t n = i0; n < N; n += stride) {
                const float d = y[o + n] - t[o + n];
                if (g) g[o + n] = d * ginv;
                accf = fmaf(d, d, accf);
            }
        }
    }
    double acc = (double)accf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        atomicAdd(loss, s * inv);
    }
}

cudaError_t launch_mse(const float* y, const float* t, float* g, int64_t C, int64_t N, int64_t ld, double* loss,
                       cudaStream_t s) {
    if (cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return cudaGetLastError();
    if (C <= 0 || N <= 0) return cudaSuccess;
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const int flat4 = (ld == N && (C * N) % 4 == 0 && al(y) && al(t) && (!g || al(g))) ? 1 : 0;
    const int bs = 256;
    const int64_t work = flat4 ? C * N / 4 : N;
    int64_t blocks = (work + bs - 1) / bs;
    if (blocks > 1216) blocks = 1216;  // a few CTAs per SM: few loss atomics
    k_mse<<<(unsigned)blocks, bs, 0, s>>>(y, t, g, C, N, ld, 1.0 / ((double)C * (double)N), loss, flat4);
    return cudaGetLastError();
}

}  // namespace tfx
