// SOS cascade (no FIR in the unit) as a warp-per-tile chunked scan.
//
// Operation (TorchFX Sec. 3, lfilter semantics): each second-order section
// y[n] = b0 x[n] + b1 x[n-1] + b2 x[n-2] - a1 y[n-1] - a2 y[n-2] (a0-normalised,
// zero initial state), sections in order, every channel independently.
//
// One warp owns a tile of 32 lanes x T samples of one channel and needs no
// CTA barrier: per section, each lane runs the 2-state recursion over its T
// samples from zero state (fused with the previous section's fix-up), a
// 5-step Kogge-Stone shuffle scan of the chunk end states with the powers
// A^1..A^16 of the chunk transfer matrix A leaves the tile aggregate in lane
// 31, and the warp resolves the tile's incoming state by a warp-parallel
// decoupled look-back over the preceding tiles of the channel (one probe per
// lane per round trip; tile transfer A^32, window transfer A^1024).  Tiles are
// handed out by an atomic ticket in time-major order, so every predecessor is
// already running.  In a training forward each lane also stores the true state
// of every section at its chunk start: the checkpoints from which the adjoint
// kernel recomputes the section outputs chunk by chunk.
#include "tfx_common.cuh"

namespace tfx {

template <int T>
__device__ __forceinline__ void warp_load(const float* row, int64_t n0, int64_t N, float (&u)[T]) {
    const float* p = row + n0;
    if (n0 + T <= N && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
        const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < T / 4; ++i) {
            const float4 v = p4[i];
            u[4 * i] = v.x;
            u[4 * i + 1] = v.y;
            u[4 * i + 2] = v.z;
            u[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < T; ++i) u[i] = (n0 + i < N) ? p[i] : 0.f;
    }
}

template <int T>
__device__ __forceinline__ void warp_store(float* row, int64_t n0, int64_t N, const float (&u)[T]) {
    float* p = row + n0;
    if (n0 + T <= N && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
        float4* p4 = reinterpret_cast<float4*>(p);
#pragma unroll
        for (int i = 0; i < T / 4; ++i) p4[i] = make_float4(u[4 * i], u[4 * i + 1], u[4 * i + 2], u[4 * i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < T; ++i)
            if (n0 + i < N) p[i] = u[i];
    }
}

template <int T, bool F64>
__global__ void __launch_bounds__(128, F64 ? 4 : 6) k_sos_warp(UnitArgs a) {
    const int lane = threadIdx.x & 31;
    unsigned tk = 0;
    if (lane == 0) tk = atomicAdd(a.sc.ticket, 1u);
    tk = __shfl_sync(0xffffffffu, tk, 0);
    const int64_t tiles = a.C * a.ntt;
    if ((int64_t)tk >= tiles) return;  // the grid is rounded up to whole CTAs
    const int64_t tile = tk;
    const int64_t c = tile % a.C;
    const int64_t tt = tile / a.C;
    const int64_t t0 = tt * (int64_t)(32 * T) + (int64_t)lane * T;
    const int S = a.k.S;

    float u[T];
    warp_load<T>(a.x + c * a.ldx, t0, a.N, u);

    float2 st = make_float2(0.f, 0.f);
    float pa1 = 0.f, pa2 = 0.f;
    for (int s = 0; s <= S; ++s) {
        const bool fix = s > 0, run = s < S;
        float b0 = 0.f, c1 = 0.f, c2 = 0.f, a1 = 0.f, a2 = 0.f;
        if (run) {
            const float* cf = a.k.coef + 8 * s;
            b0 = cf[0]; c1 = cf[1]; c2 = cf[2]; a1 = cf[3]; a2 = cf[4];
        }
        // fix-up of section s-1 (homogeneous response from its true chunk
        // start state) fused with the zero-state pass of section s
        float w1 = 0.f, w2 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            float v = u[t];
            if (fix) {
                float h;
                if (t == 0) h = st.x;
                else if (t == 1) h = fmaf(-pa1, h1, st.y);
                else h = fmaf(-pa1, h1, -pa2 * h2);
                h2 = h1;
                h1 = h;
                v += h;
            }
            if (run) {
                u[t] = fmaf(b0, v, w1);
                const float n1 = fmaf(c1, v, fmaf(-a1, w1, w2));
                w2 = fmaf(c2, v, -a2 * w1);
                w1 = n1;
            } else {
                u[t] = v;
            }
        }
        if (!run) break;
        const float4* P = a.k.pw + (size_t)s * PW_LEN;

        // inclusive scan of the chunk end states: v_l = sum_{m<=l} A^m e_{l-m}
        float2 v = make_float2(w1, w2);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float4 Pd = P[d];
            const float ox = __shfl_up_sync(0xffffffffu, v.x, d);
            const float oy = __shfl_up_sync(0xffffffffu, v.y, d);
            if (lane >= d) {
                const float2 t2 = mv2(Pd, make_float2(ox, oy));
                v.x += t2.x;
                v.y += t2.y;
            }
        }
        const float4 Pl = P[lane];
        const float px = __shfl_up_sync(0xffffffffu, v.x, 1);
        const float py = __shfl_up_sync(0xffffffffu, v.y, 1);
        const float ax = __shfl_sync(0xffffffffu, v.x, 31);
        const float ay = __shfl_sync(0xffffffffu, v.y, 31);

        // decoupled look-back, warp-parallel: lane L probes the tile L+1
        // positions back (same channel); the nearest inclusive carry ends the
        // walk, every aggregate before it contributes through powers of the
        // tile transfer T32 = A^32: win = sum_m T32^m v_(tile-1-m).
        float2 win = make_float2(0.f, 0.f);
        if (F64) {
            // the same walk with FP64 carries, FP64 powers and an FP64 window;
            // the chunk start state is formed in FP64 and rounded once
            const double4* P64 = a.k.pw64 + (size_t)s * PW_LEN;
            const double2 agg = make_double2(ax, ay);
            const bool pub = tile != a.drop_tile;
            Carry* mine = a.sc.carry + tile * S + s;
            double2 wd = make_double2(0.0, 0.0);
            if (tt == 0) {
                if (lane == 0 && pub) publish_carry64(mine, 2u, agg);
            } else {
                const double4 PL = P64[32 * lane];
                double4 Mw = make_double4(1.0, 0.0, 0.0, 1.0);
                int64_t jt0 = tt - 1;
                bool published = false;
                for (;;) {
                    const int64_t jt = jt0 - lane;
                    double2 pv = make_double2(0.0, 0.0);
                    unsigned f = 2u;
                    if (jt >= 0) f = read_carry64(a.sc.carry + (jt * a.C + c) * S + s, pv);
                    const unsigned incl_mask = __ballot_sync(0xffffffffu, f >= 2u);
                    const unsigned none_mask = __ballot_sync(0xffffffffu, f == 0u);
                    if (!published && !(incl_mask & 1u)) {
                        if (lane == 0 && pub) publish_carry64(mine, 1u, agg);
                        published = true;
                    }
                    const int first = incl_mask ? (__ffs(incl_mask) - 1) : 32;
                    const unsigned need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
                    if (none_mask & need) {
                        const int wl = __ffs(none_mask & need) - 1;
                        unsigned got = 1u;
                        if (lane == wl) {
                            double2 dummy;
                            got = wait_carry64(a.sc.carry + (jt * a.C + c) * S + s, dummy, a.status);
                        }
                        got = __shfl_sync(0xffffffffu, got, wl);
                        if (got == 0u) break;
                        continue;
                    }
                    double2 cntb = make_double2(0.0, 0.0);
                    if (lane <= first) cntb = mv2d(mm2d(Mw, PL), pv);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        cntb.x += __shfl_xor_sync(0xffffffffu, cntb.x, o);
                        cntb.y += __shfl_xor_sync(0xffffffffu, cntb.y, o);
                    }
                    wd.x += cntb.x;
                    wd.y += cntb.y;
                    if (first < 32) break;
                    Mw = mm2d(Mw, P64[1024]);
                    jt0 -= 32;
                }
                if (lane == 0 && pub) {
                    double2 incl = mv2d(P64[32], wd);
                    incl.x += agg.x;
                    incl.y += agg.y;
                    publish_carry64(mine, 2u, incl);
                }
            }
            const double2 t2d = mv2d(P64[lane], wd);
            st = (lane > 0) ? make_float2((float)((double)px + t2d.x), (float)((double)py + t2d.y))
                            : make_float2((float)t2d.x, (float)t2d.y);
        } else {
            const float2 agg = make_float2(ax, ay);
            const bool pub = tile != a.drop_tile;
            Carry* mine = a.sc.carry + tile * S + s;
            if (tt == 0) {
                if (lane == 0 && pub) publish_carry(mine, 2u, agg);
            } else {
                const float4 PL = P[32 * lane];  // T32^lane
                float4 Mw = make_float4(1.f, 0.f, 0.f, 1.f);  // T32^(32 w) for window w
                int64_t jt0 = tt - 1;  // time-tile index probed by lane 0
                bool published = false;
                for (;;) {
                    const int64_t jt = jt0 - lane;
                    float2 pv = make_float2(0.f, 0.f);
                    unsigned f = 2u;  // before the channel start: zero, inclusive
                    if (jt >= 0) f = read_carry(a.sc.carry + (jt * a.C + c) * S + s, pv);
                    unsigned incl_mask = __ballot_sync(0xffffffffu, f >= 2u);
                    unsigned none_mask = __ballot_sync(0xffffffffu, f == 0u);
                    if (!published && !(incl_mask & 1u)) {
                        // predecessor not inclusive yet: let successors use our aggregate
                        if (lane == 0 && pub) publish_carry(mine, 1u, agg);
                        published = true;
                    }
                    // lanes up to the first inclusive must all hold at least an aggregate
                    const int first = incl_mask ? (__ffs(incl_mask) - 1) : 32;
                    const unsigned need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
                    if (none_mask & need) {
                        // bounded wait on the nearest lane still empty, then re-probe
                        const int wl = __ffs(none_mask & need) - 1;
                        unsigned got = 1u;
                        if (lane == wl) {
                            float2 dummy;
                            got = wait_carry(a.sc.carry + (jt * a.C + c) * S + s, dummy, a.status);
                        }
                        got = __shfl_sync(0xffffffffu, got, wl);
                        if (got == 0u) break;  // gave up: status word records the timeout
                        continue;
                    }
                    float2 cntb = make_float2(0.f, 0.f);
                    if (lane <= first) cntb = mv2(mm2(Mw, PL), pv);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        cntb.x += __shfl_xor_sync(0xffffffffu, cntb.x, o);
                        cntb.y += __shfl_xor_sync(0xffffffffu, cntb.y, o);
                    }
                    win.x += cntb.x;
                    win.y += cntb.y;
                    if (first < 32) break;
                    Mw = mm2(Mw, P[1024]);
                    jt0 -= 32;
                }
                if (lane == 0 && pub) {
                    float2 incl = mv2(P[32], win);
                    incl.x += agg.x;
                    incl.y += agg.y;
                    publish_carry(mine, 2u, incl);
                }
            }
            // true start state of this lane's chunk
            st = (lane > 0) ? make_float2(px, py) : make_float2(0.f, 0.f);
            const float2 t2 = mv2(Pl, win);
            st.x += t2.x;
            st.y += t2.y;
        }
        // training forward: keep the chunk-start state (block-boundary checkpoint)
        if (a.ckpt) {
            const int64_t chunk = tt * 32 + lane;
            if (chunk < a.nch) a.ckpt[(c * S + s) * a.nch + chunk] = st;
        }
        pa1 = a1;
        pa2 = a2;
    }
    warp_store<T>(a.y + c * a.ldy, t0, a.N, u);
}

cudaError_t launch_sos_warp(const UnitArgs& a, cudaStream_t s) {
    const int64_t tiles = a.C * a.ntt;
    if (tiles <= 0) return cudaSuccess;
    const int64_t ctas = (tiles + 3) / 4;
    if (a.k.pw64)
        k_sos_warp<T_CHUNK, true><<<(unsigned)ctas, 128, 0, s>>>(a);
    else
        k_sos_warp<T_CHUNK, false><<<(unsigned)ctas, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tfx
