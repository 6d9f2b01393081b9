// Batched execution of many clips, each with its own shape and chain, in a
// handful of launches (the multichannel, many-clip throughput the paper's
// Sec. 4 is about, as one capturable batch).
//
// The clips are packed into one input and one output buffer (clip i at a
// fixed offset, rows of its own length).  Each clip gets an ordinary plan
// (validation, grouping into units, FP64 constants).  Clips whose chain
// composes into one FIR (the composite impulse response, as for a single
// chain) run by FFT overlap-save, all clips of one transform size in ONE
// launch.  The batch groups the other clips' units by position in their
// chain (level) and by kernel (fused cascade + short FIR, cascade only,
// FFT FIR by transform size, tensor-core FIR for FIRs a single FFT block
// cannot hold) and runs every group as ONE launch whose tiles span all of
// its units.  A CTA maps its ticket to a unit by binary search over the
// units' tile prefix sums (an FFT launch's CTA reads its unit from a per-CTA
// table built here), so each unit's tiles keep their time-major order.  Buffer
// pointers in the descriptors are offsets into the packed input, the packed
// output or the workspace, so an execution is pure pointer arithmetic on
// three base addresses: no allocation, no host synchronisation, capturable
// in a CUDA graph.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "plan_internal.cuh"

using namespace tfx;

namespace {

enum GroupKind { G_FUSED = 0, G_CASCADE = 1, G_FIR = 2, G_CHAIN_FFT = 3, G_FFT = 4 };

struct Group {
    int level = 0;
    int kind = 0;
    int nunits = 0;
    int64_t tiles = 0;
    int64_t samples = 0;  // channel-samples the group filters
    double flops = 0.0;   // algorithmic: 10 per section-sample, 2 L per FIR sample
    size_t smem = 0;
    size_t desc_off = 0, prefix_off = 0;  // in the batch's device descriptor blob
    size_t map_off = 0;                   // FFT groups: the unit of every CTA (int32)
    size_t hdr_off = 0, hdr_bytes = 0;    // workspace: ticket + flags + carries (zeroed per execution)
    std::vector<BatchUnit> units;
    std::vector<BatchFir> firs;
    std::vector<BatchFft> ffts;
    int fft_m = 0;                  // FFT groups: transform size 2^fft_m
    const float2* tw = nullptr;     // its twiddle tables (in one of the clips' plans)
    std::vector<int64_t> prefix;
};

}  // namespace

struct tfx_batch {
    int nclips = 0;
    std::vector<tfx_plan*> plans;
    std::vector<int64_t> off;  // packed offset of each clip (floats)
    int64_t total = 0;         // floats in the packed input (= output)
    std::vector<Group> groups;
    std::vector<int> identity;  // clips whose chain is empty (copied)
    char* ddesc = nullptr;
    int* dstatus = nullptr;
    size_t ws_bytes = 0;
};

namespace {

void batch_free(tfx_batch* b) {
    if (!b) return;
    if (b->ddesc || b->dstatus) cudaDeviceSynchronize();
    for (tfx_plan* p : b->plans) tfx_plan_destroy(p);
    if (b->ddesc) cudaFree(b->ddesc);
    if (b->dstatus) cudaFree(b->dstatus);
    delete b;
}

int batch_build(tfx_batch* b, const tfx_clip* clips, int32_t n, const tfx_batch_params& prm) {
    const int NB = prm.fir_nb > 0 ? prm.fir_nb : 128;
    if (NB != 64 && NB != 128 && NB != 256) return TFX_ERR_INVALID;
    // A clip whose chain composes (its cascades' response decays; see
    // compose_chain) runs as one FFT FIR of its composite response, batched
    // with every other composed clip of the same transform size in one
    // launch.  The other clips' units run grouped by level and kernel: FIRs by
    // single-block FFT overlap-save where a block holds the taps (else on the
    // tensor cores), short FIRs fused with a cascade.
    const uint32_t pflags = prm.plan_flags | TFX_PLAN_SCAN_LOOKBACK;
    if (pflags & (TFX_PLAN_SCAN_WARP_TILES | TFX_PLAN_TRAINABLE | TFX_PLAN_TEST_DROP_PUBLISH | TFX_PLAN_UNFUSED |
                  TFX_PLAN_FIR_FFT))
        return TFX_ERR_UNSUPPORTED;
    const bool compose = !(prm.plan_flags & (TFX_PLAN_NO_COMPOSE | TFX_PLAN_FIR_CUDA_CORES |
                                               TFX_PLAN_FIR_BF16_PLAIN | TFX_PLAN_FIR_BF16_SPLIT));
    b->nclips = n;
    b->plans.assign(n, nullptr);
    b->off.resize(n);
    int64_t off = 0;
    for (int i = 0; i < n; ++i) {
        const tfx_clip& c = clips[i];
        if (c.C < 0 || c.N < 0) return TFX_ERR_INVALID;
        b->off[i] = off;
        if (c.C > 0 && c.N > INT64_MAX / c.C) return TFX_ERR_INVALID;
        off += c.C * c.N;
        // the batched cascade kernel carries in FP32: no FP64-carry routing
        int rc = TFX_OK;
        if (compose && c.C > 0 && c.N > 0) {
            rc = plan_create_ex(&b->plans[i], c.C, c.N, c.N, c.st, c.nst, prm.plan_flags, prm.tc_min_taps, false,
                                prm.fft_m);
            if (rc != TFX_OK) return rc;
            if (b->plans[i]->use_chain) continue;
            tfx_plan_destroy(b->plans[i]);
            b->plans[i] = nullptr;
        }
        rc = plan_create_ex(&b->plans[i], c.C, c.N, c.N > 0 ? c.N : 1, c.st, c.nst, pflags, prm.tc_min_taps, false);
        if (rc != TFX_OK) return rc;
        // a partitioned FFT FIR (two launches and a spectra workspace) is not
        // batched: such a clip's FIRs go to the tensor cores
        bool partitioned = false;
        for (const HostUnit& u : b->plans[i]->units) partitioned = partitioned || (u.fft && u.fft_P > 0);
        if (partitioned) {
            tfx_plan_destroy(b->plans[i]);
            b->plans[i] = nullptr;
            rc = plan_create_ex(&b->plans[i], c.C, c.N, c.N > 0 ? c.N : 1, c.st, c.nst, pflags | TFX_PLAN_FIR_TC,
                                prm.tc_min_taps, false);
            if (rc != TFX_OK) return rc;
        }
    }
    b->total = off;
    if (cudaMalloc(&b->dstatus, sizeof(int)) != cudaSuccess) return TFX_ERR_NOMEM;
    if (cudaMemset(b->dstatus, 0, sizeof(int)) != cudaSuccess) return TFX_ERR_CUDA;

    // workspace: per clip its unit-to-unit intermediates, then per group its
    // header (ticket + tile flags + carries) and its FIR-input tails
    size_t ws = 0;
    std::vector<std::vector<size_t>> inter(n);  // byte offsets of the intermediates of clip i
    for (int i = 0; i < n; ++i) {
        const tfx_plan* p = b->plans[i];
        const int nu = (int)p->units.size();
        if (p->C == 0 || p->N == 0 || p->use_chain) continue;
        if (nu == 0) b->identity.push_back(i);
        const int nbuf = nu > 2 ? 2 : (nu == 2 ? 1 : 0);
        for (int k = 0; k < nbuf; ++k) {
            inter[i].push_back(ws);
            ws = align_up(ws + (size_t)p->C * p->N * sizeof(float));
        }
    }
    // composed clips: one group per transform size
    for (int m = 10; m <= 14; ++m) {
        Group g;
        g.kind = G_CHAIN_FFT;
        g.fft_m = m;
        g.prefix.push_back(0);
        for (int i = 0; i < n; ++i) {
            tfx_plan* p = b->plans[i];
            if (!p->use_chain || p->chain.fft_m != m) continue;
            const HostUnit& u = p->chain;
            BatchFft f{};
            f.x_sel = 0;
            f.y_sel = 1;
            f.x_off = b->off[i];
            f.y_off = b->off[i];
            f.C = p->C;
            f.N = p->N;
            f.L = u.L;
            f.B = u.fft_B;
            f.nbpc = (p->N + u.fft_B - 1) / u.fft_B;
            f.nb = p->C * f.nbpc;
            f.H = reinterpret_cast<const float2*>(p->dconst + u.off_H);
            if (!g.tw) g.tw = reinterpret_cast<const float2*>(p->dconst + u.off_tw);
            g.ffts.push_back(f);
            g.tiles += (f.nb + 1) / 2;
            g.prefix.push_back(g.tiles);
            g.samples += p->C * p->N;
            const double Mm = (double)(1 << m);
            g.flops += (10.0 * Mm * m + 6.0 * Mm) / (2.0 * u.fft_B) * (double)(p->C * p->N);
        }
        g.nunits = (int)g.ffts.size();
        if (g.nunits == 0) continue;
        if (g.tiles > (int64_t)INT32_MAX) return TFX_ERR_UNSUPPORTED;
        b->groups.push_back(g);
    }
    int maxlev = 0;
    for (int i = 0; i < n; ++i)
        if (b->plans[i]->C > 0 && b->plans[i]->N > 0 && !b->plans[i]->use_chain)
            maxlev = std::max(maxlev, (int)b->plans[i]->units.size());
    for (int lev = 0; lev < maxlev; ++lev) {
        Group g[3];
        for (int k = 0; k < 3; ++k) {
            g[k].level = lev;
            g[k].kind = k;
            g[k].prefix.push_back(0);
        }
        Group gf[5];  // FFT FIR units by transform size 2^(10 + k)
        for (int k = 0; k < 5; ++k) {
            gf[k].level = lev;
            gf[k].kind = G_FFT;
            gf[k].fft_m = 10 + k;
            gf[k].prefix.push_back(0);
        }
        // header offsets are relative to the group's header start for now
        size_t hdr[3] = {ALIGN, ALIGN, ALIGN};
        size_t tails[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i) {
            tfx_plan* p = b->plans[i];
            const int nu = (int)p->units.size();
            if (p->C == 0 || p->N == 0 || lev >= nu || p->use_chain) continue;
            HostUnit u = p->units[lev];
            // where this unit reads and writes: batch input/output or an intermediate
            const int ib = lev == 0 ? -1 : ((lev - 1) & 1);
            const int ob = lev == nu - 1 ? -1 : (lev & 1);
            const int x_sel = ib < 0 ? 0 : 2, y_sel = ob < 0 ? 1 : 2;
            const int64_t x_off = ib < 0 ? b->off[i] : (int64_t)(inter[i][ib] / sizeof(float));
            const int64_t y_off = ob < 0 ? b->off[i] : (int64_t)(inter[i][ob] / sizeof(float));
            if (u.fft) {  // single-block (partitioned units were sent to the tensor cores)
                int m = 0;
                while ((1 << m) < u.fft_M) ++m;
                if (u.fft_P != 0 || m < 10 || m > 14) return TFX_ERR_UNSUPPORTED;
                Group& gr = gf[m - 10];
                BatchFft f{};
                f.x_sel = x_sel;
                f.y_sel = y_sel;
                f.x_off = x_off;
                f.y_off = y_off;
                f.C = p->C;
                f.N = p->N;
                f.L = u.L;
                f.B = u.fft_B;
                f.nbpc = (p->N + u.fft_B - 1) / u.fft_B;
                f.nb = p->C * f.nbpc;
                f.H = reinterpret_cast<const float2*>(p->dconst + u.off_H);
                if (!gr.tw) gr.tw = reinterpret_cast<const float2*>(p->dconst + u.off_tw);
                gr.ffts.push_back(f);
                gr.tiles += (f.nb + 1) / 2;
                gr.prefix.push_back(gr.tiles);
                gr.samples += p->C * p->N;
                gr.flops += 2.0 * u.L * (double)(p->C * p->N);
                continue;
            }
            if (u.tc) {
                tc_geometry(u, NB);
                if (u.tc_smem > SMEM_MAX) return TFX_ERR_UNSUPPORTED;  // tap tables too large to batch
                BatchFir f{};
                FirTcArgs& a = f.a;
                a.C = p->C;
                a.N = p->N;
                a.ldx = p->N;
                a.ldy = p->N;
                a.ntt = (p->N + 128 * u.NB - 1) / (128 * u.NB);
                a.L = u.L;
                a.W = u.W;
                a.nK = u.nK;
                a.NB = u.NB;
                a.rows = u.rows;
                a.tmem_cols = u.tmem_cols;
                a.a_chunks = u.a_chunks;
                a.mode = u.tc_mode;
                a.persistent = 0;
                a.grid = 0;
                a.tap_unscale = u.tap_unscale;
                a.a_hi = reinterpret_cast<const uint4*>(p->dconst + u.off_ahi);
                a.a_lo = reinterpret_cast<const uint4*>(p->dconst + u.off_alo);
                a.status = b->dstatus;
                f.x_sel = x_sel;
                f.y_sel = y_sel;
                f.x_off = x_off;
                f.y_off = y_off;
                g[G_FIR].samples += p->C * p->N;
                g[G_FIR].flops += 2.0 * u.L * (double)(p->C * p->N);
                g[G_FIR].firs.push_back(f);
                g[G_FIR].tiles += a.C * a.ntt;
                g[G_FIR].prefix.push_back(g[G_FIR].tiles);
                g[G_FIR].smem = std::max(g[G_FIR].smem, fir_tc_smem_bytes(a));
                continue;
            }
            const int k = u.L > 0 ? G_FUSED : G_CASCADE;
            BatchUnit bu{};
            UnitArgs& a = bu.a;
            a.C = p->C;
            a.N = p->N;
            a.ldx = p->N;
            a.ldy = p->N;
            a.ntt = u.ntt;
            a.k.S = u.S;
            a.k.L = u.L;
            a.k.H = u.L > 0 ? u.L - 1 : 0;
            a.k.nkb = u.nkb;
            a.k.gain = 1.0f;
            a.k.coef = reinterpret_cast<const float*>(p->dconst + u.off_coef);
            a.k.pw = reinterpret_cast<const float4*>(p->dconst + u.off_pw);
            a.k.taps = reinterpret_cast<const float*>(p->dconst + u.off_taps);
            a.sc.tail_len = u.tail_len;
            a.status = b->dstatus;
            a.drop_tile = -1;
            const int64_t tiles = p->C * u.ntt;
            bu.x_sel = x_sel;
            bu.y_sel = y_sel;
            bu.x_off = x_off;
            bu.y_off = y_off;
            bu.flags_off = (int64_t)hdr[k];
            hdr[k] = align_up(hdr[k] + (size_t)tiles * sizeof(unsigned));
            bu.carry_off = (int64_t)hdr[k];
            hdr[k] = align_up(hdr[k] + (size_t)tiles * u.S * sizeof(Carry));
            bu.tails_off = (int64_t)tails[k];
            tails[k] = align_up(tails[k] + (size_t)tiles * u.tail_len * sizeof(float));
            g[k].samples += p->C * p->N;
            g[k].flops += (10.0 * u.S + 2.0 * u.L) * (double)(p->C * p->N);
            g[k].units.push_back(bu);
            g[k].tiles += tiles;
            g[k].prefix.push_back(g[k].tiles);
            if (u.L > 0) {
                UnitConst kc{};
                kc.S = u.S;
                kc.L = u.L;
                kc.H = u.L - 1;
                kc.nkb = u.nkb;
                g[k].smem = std::max(g[k].smem, unit_smem_bytes(kc));
            }
        }
        for (int k = 0; k < 3; ++k) {
            Group& gr = g[k];
            gr.nunits = k == G_FIR ? (int)gr.firs.size() : (int)gr.units.size();
            if (gr.nunits == 0) continue;
            if (gr.tiles > (int64_t)INT32_MAX) return TFX_ERR_UNSUPPORTED;
            // place the group's header and tails in the workspace
            gr.hdr_off = ws;
            gr.hdr_bytes = k == G_FIR ? 0 : hdr[k];
            ws = align_up(ws + gr.hdr_bytes);
            const size_t tails_base = ws;
            ws = align_up(ws + tails[k]);
            for (BatchUnit& bu : gr.units) {
                bu.flags_off += (int64_t)gr.hdr_off;
                bu.carry_off += (int64_t)gr.hdr_off;
                bu.tails_off += (int64_t)tails_base;
            }
            if (k == G_FUSED && prepare_unit_batched(gr.smem) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
            if (k == G_FIR && prepare_fir_tc_batched(gr.smem) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
            b->groups.push_back(gr);
        }
        for (Group& gr : gf) {
            gr.nunits = (int)gr.ffts.size();
            if (gr.nunits == 0) continue;
            if (gr.tiles > (int64_t)INT32_MAX) return TFX_ERR_UNSUPPORTED;
            b->groups.push_back(gr);
        }
    }
    b->ws_bytes = ws;

    // descriptors and prefix sums of every group in one device blob
    size_t blob = 0;
    auto desc_bytes = [](const Group& gr) {
        return gr.kind == G_FIR                             ? gr.firs.size() * sizeof(BatchFir)
               : gr.kind == G_CHAIN_FFT || gr.kind == G_FFT ? gr.ffts.size() * sizeof(BatchFft)
                                                            : gr.units.size() * sizeof(BatchUnit);
    };
    auto is_fft = [](const Group& gr) { return gr.kind == G_CHAIN_FFT || gr.kind == G_FFT; };
    for (Group& gr : b->groups) {
        gr.desc_off = blob;
        blob = align_up(blob + desc_bytes(gr));
        gr.prefix_off = blob;
        blob = align_up(blob + gr.prefix.size() * sizeof(int64_t));
        if (is_fft(gr)) {
            gr.map_off = blob;
            blob = align_up(blob + (size_t)gr.tiles * sizeof(int32_t));
        }
    }
    if (blob > 0) {
        std::vector<char> host(blob, 0);
        for (const Group& gr : b->groups) {
            if (gr.kind == G_FIR)
                std::memcpy(host.data() + gr.desc_off, gr.firs.data(), gr.firs.size() * sizeof(BatchFir));
            else if (gr.kind == G_CHAIN_FFT || gr.kind == G_FFT)
                std::memcpy(host.data() + gr.desc_off, gr.ffts.data(), gr.ffts.size() * sizeof(BatchFft));
            else
                std::memcpy(host.data() + gr.desc_off, gr.units.data(), gr.units.size() * sizeof(BatchUnit));
            std::memcpy(host.data() + gr.prefix_off, gr.prefix.data(), gr.prefix.size() * sizeof(int64_t));
            if (is_fft(gr)) {
                int32_t* map = reinterpret_cast<int32_t*>(host.data() + gr.map_off);
                for (int u = 0; u < gr.nunits; ++u)
                    for (int64_t k = gr.prefix[u]; k < gr.prefix[u + 1]; ++k) map[k] = u;
            }
        }
        if (cudaMalloc(&b->ddesc, blob) != cudaSuccess) return TFX_ERR_NOMEM;
        if (cudaMemcpy(b->ddesc, host.data(), blob, cudaMemcpyHostToDevice) != cudaSuccess) return TFX_ERR_CUDA;
    }
    return TFX_OK;
}

int run_group(tfx_batch* b, const Group& gr, const BatchBases& bases, char* w, cudaStream_t s) {
    const int64_t* prefix = reinterpret_cast<const int64_t*>(b->ddesc + gr.prefix_off);
    if (gr.kind == G_CHAIN_FFT || gr.kind == G_FFT)
        return launch_fir_fft_batched(gr.fft_m, reinterpret_cast<const BatchFft*>(b->ddesc + gr.desc_off), prefix,
                                      reinterpret_cast<const int32_t*>(b->ddesc + gr.map_off), gr.nunits, gr.tiles,
                                      bases, gr.tw, s) == cudaSuccess
                   ? TFX_OK
                   : TFX_ERR_CUDA;
    if (gr.kind == G_FIR)
        return launch_fir_tc_batched(reinterpret_cast<const BatchFir*>(b->ddesc + gr.desc_off), prefix, gr.nunits,
                                     gr.tiles, bases, gr.smem, s) == cudaSuccess
                   ? TFX_OK
                   : TFX_ERR_CUDA;
    if (cudaMemsetAsync(w + gr.hdr_off, 0, gr.hdr_bytes, s) != cudaSuccess) return TFX_ERR_CUDA;
    return launch_unit_batched(gr.kind == G_FUSED, reinterpret_cast<const BatchUnit*>(b->ddesc + gr.desc_off),
                               prefix, gr.nunits, gr.tiles, reinterpret_cast<unsigned*>(w + gr.hdr_off), bases,
                               gr.smem, s) == cudaSuccess
               ? TFX_OK
               : TFX_ERR_CUDA;
}

}  // namespace

extern "C" {

int tfx_batch_create(tfx_batch** out, const tfx_clip* clips, int32_t nclips, const tfx_batch_params* prm) {
    if (!out) return TFX_ERR_INVALID;
    *out = nullptr;
    if (nclips < 0 || (nclips > 0 && !clips)) return TFX_ERR_INVALID;
    tfx_batch_params p{};
    if (prm) p = *prm;
    tfx_batch* b = new (std::nothrow) tfx_batch();
    if (!b) return TFX_ERR_NOMEM;
    const int rc = batch_build(b, clips, nclips, p);
    if (rc != TFX_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return TFX_OK;
}

int64_t tfx_batch_total_samples(const tfx_batch* b) { return b ? b->total : -1; }

int64_t tfx_batch_clip_offset(const tfx_batch* b, int32_t i) {
    if (!b || i < 0 || i >= b->nclips) return -1;
    return b->off[i];
}

size_t tfx_batch_workspace_size(const tfx_batch* b) { return b ? b->ws_bytes : 0; }

int tfx_batch_launch_count(const tfx_batch* b) {
    if (!b) return -1;
    return (int)b->groups.size() + (int)b->identity.size();
}

int tfx_batch_execute(tfx_batch* b, const float* x, float* y, void* ws, size_t ws_bytes, tfx_stream stream) {
    if (!b) return TFX_ERR_INVALID;
    if (b->total == 0) return TFX_OK;
    if (!x || !y) return TFX_ERR_INVALID;
    {
        const char* xb = reinterpret_cast<const char*>(x);
        const char* yb = reinterpret_cast<const char*>(y);
        const size_t span = (size_t)b->total * sizeof(float);
        if (xb < yb + span && yb < xb + span) return TFX_ERR_INVALID;  // no in-place batches
    }
    if (b->ws_bytes > 0 && (!ws || ws_bytes < b->ws_bytes || reinterpret_cast<uintptr_t>(ws) % ALIGN != 0))
        return TFX_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    BatchBases bases{x, y, reinterpret_cast<float*>(w)};
    for (int i : b->identity) {
        const tfx_plan* p = b->plans[i];
        if (cudaMemcpyAsync(y + b->off[i], x + b->off[i], (size_t)p->C * p->N * sizeof(float),
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return TFX_ERR_CUDA;
    }
    for (const Group& gr : b->groups) {
        const int rc = run_group(b, gr, bases, w, s);
        if (rc != TFX_OK) return rc;
    }
    return TFX_OK;
}

int tfx_batch_clip_info(const tfx_batch* b, int32_t i, int32_t* composed, int32_t* taps, int32_t* fft_m) {
    if (!b || i < 0 || i >= b->nclips || !b->plans[i]) return TFX_ERR_INVALID;
    const tfx_plan* p = b->plans[i];
    if (composed) *composed = p->use_chain ? 1 : 0;
    if (taps) *taps = p->use_chain ? p->chain.L : 0;
    if (fft_m) *fft_m = p->use_chain ? p->chain.fft_m : 0;
    return TFX_OK;
}

int tfx_batch_group_count(const tfx_batch* b) { return b ? (int)b->groups.size() : -1; }

int tfx_batch_group_info(const tfx_batch* b, int32_t g, int32_t* kind, int32_t* level, int64_t* tiles,
                         int64_t* samples, double* flops) {
    if (!b || g < 0 || g >= (int)b->groups.size()) return TFX_ERR_INVALID;
    const Group& gr = b->groups[g];
    if (kind) *kind = gr.kind;
    if (level) *level = gr.level;
    if (tiles) *tiles = gr.tiles;
    if (samples) *samples = gr.samples;
    if (flops) *flops = gr.flops;
    return TFX_OK;
}

int tfx_batch_execute_group(tfx_batch* b, int32_t g, const float* x, float* y, void* ws, size_t ws_bytes,
                            tfx_stream stream) {
    if (!b || g < 0 || g >= (int)b->groups.size() || !x || !y) return TFX_ERR_INVALID;
    if (b->ws_bytes > 0 && (!ws || ws_bytes < b->ws_bytes || reinterpret_cast<uintptr_t>(ws) % ALIGN != 0))
        return TFX_ERR_WORKSPACE;
    char* w = static_cast<char*>(ws);
    BatchBases bases{x, y, reinterpret_cast<float*>(w)};
    return run_group(b, b->groups[g], bases, w, reinterpret_cast<cudaStream_t>(stream));
}

int tfx_batch_get_error(tfx_batch* b) {
    if (!b || !b->dstatus) return TFX_ERR_INVALID;
    if (cudaDeviceSynchronize() != cudaSuccess) return TFX_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, b->dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TFX_ERR_CUDA;
    if (v != 0 && cudaMemset(b->dstatus, 0, sizeof(int)) != cudaSuccess) return TFX_ERR_CUDA;
    return v;
}

void tfx_batch_destroy(tfx_batch* b) { batch_free(b); }

}  // extern "C"
