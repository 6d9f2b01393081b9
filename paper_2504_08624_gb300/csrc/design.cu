// Filter design and plan-constant updates on the GPU, in FP64.
//
// k_design computes second-order sections from design parameters, one
// thread per filter: Butterworth low/high-pass and Chebyshev-I low-pass by
// the bilinear transform of the analog prototype with the cutoff prewarped
// to tan(pi fc / fs) (TorchFX Sec. 3 designs its IIR filters from such
// parameters), sections ordered by increasing pole radius, each with its
// zeros at z = -1 (low) or +1 (high) and unit gain at DC (low) or Nyquist
// (high); RBJ peaking and shelving biquads; and the biquad whose poles are
// parameterised by radius r = rmin + rspan sigmoid(rho) and angle
// theta = pi sigmoid(phi) (the learnable cascade).  Rows are written raw
// (b0 b1 b2 a0 a1 a2, a0 = 1).
//
// k_update_sections recomputes a plan's section constants from raw FP64 rows
// in device memory: the a0 normalisation, the c-form coefficients, and the
// chunk-transfer powers A^k (k = 0..1024, FP32 and, for FP64-carry cascades,
// FP64), each power by binary exponentiation of A = M^chunk.  Designs and
// coefficient updates then never leave the device (no host round trip in a
// training loop).
#include <cmath>

#include "plan_internal.cuh"

using namespace tfx;

namespace {

struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }

constexpr int DESIGN_MAX_ORDER = 16;

// one section from a digital pole (complex: conjugate pair; real: first
// order), zeros at `zero`, unit gain at z = ug (+1 DC, -1 Nyquist)
__device__ void section_from_pole(cplx z, double zero, double ug, double* row) {
    double a0 = 1.0, a1, a2, b0 = 1.0, b1, b2;
    if (fabs(z.im) > 0.0) {
        a1 = -2.0 * z.re;
        a2 = cabs2(z);
        b1 = -2.0 * zero;
        b2 = zero * zero;
    } else {
        a1 = -z.re;
        a2 = 0.0;
        b1 = -zero;
        b2 = 0.0;
    }
    const double num = b0 + b1 * ug + b2 * ug * ug;
    const double den = a0 + a1 * ug + a2 * ug * ug;
    const double g = den / num;
    row[0] = b0 * g;
    row[1] = b1 * g;
    row[2] = b2 * g;
    row[3] = a0;
    row[4] = a1;
    row[5] = a2;
}

// analog prototype poles (upper half plane and real), scaled, bilinear,
// sorted by radius (stable), written as sections
__device__ void poles_to_sections(const cplx* analog, int order, double zero, double ug, double* rows) {
    cplx z[DESIGN_MAX_ORDER];
    int nz = 0;
    for (int k = 0; k < order; ++k) {
        const cplx p = analog[k];
        if (p.im > 1e-14 || fabs(p.im) <= 1e-14) {
            const cplx q = {p.im > 1e-14 ? p.re : p.re, p.im > 1e-14 ? p.im : 0.0};
            z[nz++] = cdiv({1.0 + q.re, q.im}, {1.0 - q.re, -q.im});  // z = (1 + s) / (1 - s)
        }
    }
    for (int i = 1; i < nz; ++i) {  // stable insertion sort by |z|
        const cplx v = z[i];
        const double key = cabs2(v);
        int j = i - 1;
        while (j >= 0 && cabs2(z[j]) > key) {
            z[j + 1] = z[j];
            --j;
        }
        z[j + 1] = v;
    }
    for (int i = 0; i < nz; ++i) section_from_pole(z[i], zero, ug, rows + 6 * i);
}

__global__ void k_design(const tfx_design* __restrict__ specs, int n, const int64_t* __restrict__ row_off,
                         double* __restrict__ rows, int* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const tfx_design d = specs[i];
    double* out = rows + 6 * row_off[i];
    const double pi = 3.14159265358979323846;
    switch (d.kind) {
        case TFX_DESIGN_BUTTER_LOW:
        case TFX_DESIGN_BUTTER_HIGH:
        case TFX_DESIGN_CHEBY1_LOW: {
            const int order = d.order;
            if (order < 1 || order > DESIGN_MAX_ORDER || !(d.f1 > 0.0 && d.f1 < d.fs / 2)) {
                atomicCAS(status, 0, (int)TFX_ERR_INVALID);
                return;
            }
            const double K = tan(pi * d.f1 / d.fs);
            cplx analog[DESIGN_MAX_ORDER];
            if (d.kind == TFX_DESIGN_CHEBY1_LOW) {
                const double eps = sqrt(pow(10.0, d.p1 / 10.0) - 1.0);
                const double mu = asinh(1.0 / eps) / order;
                for (int k = 0; k < order; ++k) {
                    const double th = pi * (2 * k + 1) / (2.0 * order);
                    analog[k] = {-sinh(mu) * sin(th) * K, cosh(mu) * cos(th) * K};
                }
            } else {
                for (int k = 0; k < order; ++k) {
                    const double ang = pi * (2 * k + order + 1) / (2.0 * order);
                    const cplx q = {cos(ang), sin(ang)};
                    analog[k] = d.kind == TFX_DESIGN_BUTTER_LOW ? cplx{K * q.re, K * q.im} : cdiv({K, 0.0}, q);
                }
            }
            const bool high = d.kind == TFX_DESIGN_BUTTER_HIGH;
            poles_to_sections(analog, order, high ? 1.0 : -1.0, high ? -1.0 : 1.0, out);
            if (d.kind == TFX_DESIGN_CHEBY1_LOW && order % 2 == 0) {
                const double g = pow(10.0, -d.p1 / 20.0);  // even order: DC at the ripple floor
                out[0] *= g;
                out[1] *= g;
                out[2] *= g;
            }
            break;
        }
        case TFX_DESIGN_PEAKING: {
            const double A = pow(10.0, d.p2 / 40.0), w0 = 2.0 * pi * d.f1 / d.fs;
            const double alpha = sin(w0) / (2.0 * d.p1), cw = cos(w0);
            const double a0 = 1.0 + alpha / A;
            out[0] = (1.0 + alpha * A) / a0;
            out[1] = -2.0 * cw / a0;
            out[2] = (1.0 - alpha * A) / a0;
            out[3] = 1.0;
            out[4] = -2.0 * cw / a0;
            out[5] = (1.0 - alpha / A) / a0;
            break;
        }
        case TFX_DESIGN_LOW_SHELF:
        case TFX_DESIGN_HIGH_SHELF: {
            const double A = pow(10.0, d.p1 / 40.0), w0 = 2.0 * pi * d.f1 / d.fs, cw = cos(w0);
            const double slope = d.p2 > 0.0 ? d.p2 : 1.0;
            const double alpha = sin(w0) / 2.0 * sqrt((A + 1.0 / A) * (1.0 / slope - 1.0) + 2.0);
            const double q = 2.0 * sqrt(A) * alpha;
            double b[3], a[3];
            if (d.kind == TFX_DESIGN_LOW_SHELF) {
                b[0] = A * ((A + 1) - (A - 1) * cw + q);
                b[1] = 2 * A * ((A - 1) - (A + 1) * cw);
                b[2] = A * ((A + 1) - (A - 1) * cw - q);
                a[0] = (A + 1) + (A - 1) * cw + q;
                a[1] = -2 * ((A - 1) + (A + 1) * cw);
                a[2] = (A + 1) + (A - 1) * cw - q;
            } else {
                b[0] = A * ((A + 1) + (A - 1) * cw + q);
                b[1] = -2 * A * ((A - 1) + (A + 1) * cw);
                b[2] = A * ((A + 1) + (A - 1) * cw - q);
                a[0] = (A + 1) - (A - 1) * cw + q;
                a[1] = 2 * ((A - 1) - (A + 1) * cw);
                a[2] = (A + 1) - (A - 1) * cw - q;
            }
            out[0] = b[0] / a[0];
            out[1] = b[1] / a[0];
            out[2] = b[2] / a[0];
            out[3] = 1.0;
            out[4] = a[1] / a[0];
            out[5] = a[2] / a[0];
            break;
        }
        case TFX_DESIGN_BIQUAD_POLAR: {
            const double r = d.f1 + d.f2 / (1.0 + exp(-d.p1));  // f1 = rmin, f2 = rspan, p1 = rho
            const double th = pi / (1.0 + exp(-d.p2));          // p2 = phi
            out[0] = d.b[0];
            out[1] = d.b[1];
            out[2] = d.b[2];
            out[3] = 1.0;
            out[4] = -2.0 * r * cos(th);
            out[5] = r * r;
            break;
        }
        default:
            atomicCAS(status, 0, (int)TFX_ERR_INVALID);
    }
}

// Section constants of one plan section from its raw row: grid (sections),
// block PW_LEN-ish threads, thread k writes A^k.
struct SecUpdate {
    int64_t row;        // raw row index in a compact rows array (6 doubles per row)
    int64_t flat;       // offset of the raw row in the chain's flat coefficient array
    float* coef;        // [8]
    float4* pw;         // [PW_LEN]
    double4* pw64;      // [PW_LEN] or null
    double* raw_copy;   // trainable plans: the raw row for the a0 chain rule, or null
    float* plain;       // [8]: the plain path's copy of the section constants
    int chunk;          // samples per thread of the unit's scan
};

// One FIR stage's FP32 taps from the flat coefficient array: the CUDA-core
// and plain-path copies (zero-padded to `lpad` and `L`).
struct FirUpdate {
    int64_t flat;
    int L, lpad;
    float* taps;
    float* plain;
};

__global__ void k_update_fir_taps(const FirUpdate* __restrict__ firs, const double* __restrict__ coef) {
    const FirUpdate f = firs[blockIdx.x];
    for (int k = threadIdx.x; k < f.lpad; k += blockDim.x) {
        const float v = k < f.L ? (float)coef[f.flat + k] : 0.f;
        f.taps[k] = v;
        if (k < f.L) f.plain[k] = v;
    }
}

__global__ void k_update_sections(const SecUpdate* __restrict__ secs, const double* __restrict__ rows, int flat,
                                  int* __restrict__ status) {
    const SecUpdate su = secs[blockIdx.x];
    const double* r = rows + (flat ? su.flat : 6 * su.row);
    if (r[3] == 0.0 || !isfinite(r[0] + r[1] + r[2] + r[3] + r[4] + r[5])) {
        if (threadIdx.x == 0) atomicCAS(status, 0, (int)TFX_ERR_INVALID);
        return;
    }
    const double inv = 1.0 / r[3];
    const double b0 = r[0] * inv, b1 = r[1] * inv, b2 = r[2] * inv, a1 = r[4] * inv, a2 = r[5] * inv;
    if (!(fabs(a2) < 1.0 && fabs(a1) < 1.0 + a2)) {
        if (threadIdx.x == 0) atomicCAS(status, 0, (int)TFX_ERR_UNSTABLE);
        return;
    }
    if (threadIdx.x == 0) {
        su.coef[0] = (float)b0;
        su.coef[1] = (float)(b1 - a1 * b0);
        su.coef[2] = (float)(b2 - a2 * b0);
        su.coef[3] = (float)a1;
        su.coef[4] = (float)a2;
        su.coef[5] = (float)(a1 * b2 - a2 * b1);
        if (su.raw_copy)
            for (int j = 0; j < 6; ++j) su.raw_copy[j] = r[j];
        for (int j = 0; j < 6; ++j) su.plain[j] = su.coef[j];
    }
    // A = M^chunk, M = [[-a1, 1], [-a2, 0]] (one-sample transfer of the c-form state)
    double m00 = -a1, m01 = 1.0, m10 = -a2, m11 = 0.0;
    double A00 = 1.0, A01 = 0.0, A10 = 0.0, A11 = 1.0;
    for (int e = su.chunk; e > 0; e >>= 1) {
        if (e & 1) {
            const double t00 = A00 * m00 + A01 * m10, t01 = A00 * m01 + A01 * m11;
            const double t10 = A10 * m00 + A11 * m10, t11 = A10 * m01 + A11 * m11;
            A00 = t00; A01 = t01; A10 = t10; A11 = t11;
        }
        const double s00 = m00 * m00 + m01 * m10, s01 = m00 * m01 + m01 * m11;
        const double s10 = m10 * m00 + m11 * m10, s11 = m10 * m01 + m11 * m11;
        m00 = s00; m01 = s01; m10 = s10; m11 = s11;
    }
    for (int k = threadIdx.x; k < PW_LEN; k += blockDim.x) {
        double P00 = 1.0, P01 = 0.0, P10 = 0.0, P11 = 1.0;
        double q00 = A00, q01 = A01, q10 = A10, q11 = A11;
        for (int e = k; e > 0; e >>= 1) {
            if (e & 1) {
                const double t00 = P00 * q00 + P01 * q10, t01 = P00 * q01 + P01 * q11;
                const double t10 = P10 * q00 + P11 * q10, t11 = P10 * q01 + P11 * q11;
                P00 = t00; P01 = t01; P10 = t10; P11 = t11;
            }
            const double s00 = q00 * q00 + q01 * q10, s01 = q00 * q01 + q01 * q11;
            const double s10 = q10 * q00 + q11 * q10, s11 = q10 * q01 + q11 * q11;
            q00 = s00; q01 = s01; q10 = s10; q11 = s11;
        }
        su.pw[k] = make_float4((float)P00, (float)P01, (float)P10, (float)P11);
        if (su.pw64) su.pw64[k] = make_double4(P00, P01, P10, P11);
    }
}

}  // namespace

extern "C" {

int tfx_design_sections(const tfx_design* spec) {
    if (!spec) return -1;
    switch (spec->kind) {
        case TFX_DESIGN_BUTTER_LOW:
        case TFX_DESIGN_BUTTER_HIGH:
        case TFX_DESIGN_CHEBY1_LOW:
            if (spec->order < 1 || spec->order > DESIGN_MAX_ORDER) return -1;
            return spec->order / 2 + spec->order % 2;
        case TFX_DESIGN_PEAKING:
        case TFX_DESIGN_LOW_SHELF:
        case TFX_DESIGN_HIGH_SHELF:
        case TFX_DESIGN_BIQUAD_POLAR:
            return 1;
        default:
            return -1;
    }
}

int tfx_design_device(const tfx_design* specs, int32_t n, const int64_t* row_off, double* rows, int* status,
                      tfx_stream stream) {
    if (n < 0 || (n > 0 && (!specs || !row_off || !rows || !status))) return TFX_ERR_INVALID;
    if (n == 0) return TFX_OK;
    k_design<<<(unsigned)((n + 127) / 128), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(specs, n, row_off,
                                                                                              rows, status);
    return cudaGetLastError() == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
}

}  // extern "C"

namespace {

// Plain-path constants of every chain stage, by the stage's offset in the
// flat coefficient array (stages in order; SOS: 6 values per row, FIR: n).
std::vector<std::pair<int64_t, float*>> plain_by_flat(tfx_plan* p) {
    std::vector<std::pair<int64_t, float*>> out;
    int64_t off = 0;
    for (const PlainStage& st : p->plain) {
        float* base = reinterpret_cast<float*>(p->dconst + st.off);
        if (st.kind == TFX_STAGE_SOS) {
            for (int r = 0; r < st.n; ++r) out.push_back({off + 6 * r, base + 8 * r});
            off += 6 * (int64_t)st.n;
        } else {
            out.push_back({off, base});
            off += st.n;
        }
    }
    return out;
}

float* plain_at(const std::vector<std::pair<int64_t, float*>>& m, int64_t flat) {
    for (const auto& e : m)
        if (e.first == flat) return e.second;
    return nullptr;
}

// The per-section (and per-FIR) update descriptors, built and uploaded once
// (host-synchronous); every update after that is a few launches.
int build_update_descriptors(tfx_plan* p) {
    if (p->dsec || p->nsec == 0) return TFX_OK;
    const auto pm = plain_by_flat(p);
    std::vector<SecUpdate> v;
    std::vector<FirUpdate> f;
    int64_t row = 0;
    for (HostUnit& u : p->units) {
        for (int k = 0; k < u.S; ++k) {
            SecUpdate su{};
            su.row = row++;
            su.flat = u.dst[k];
            su.coef = reinterpret_cast<float*>(p->dconst + u.off_coef) + 8 * k;
            su.pw = reinterpret_cast<float4*>(p->dconst + u.off_pw) + (size_t)k * PW_LEN;
            su.pw64 = u.hiq ? reinterpret_cast<double4*>(p->dconst + u.off_pw64) + (size_t)k * PW_LEN : nullptr;
            su.raw_copy = p->train ? reinterpret_cast<double*>(p->dconst + u.off_raw) + 6 * k : nullptr;
            su.plain = plain_at(pm, su.flat);
            su.chunk = (u.L == 0 && !u.warp) ? T_CASCADE : T_CHUNK;
            if (!su.plain) return TFX_ERR_INVALID;
            v.push_back(su);
        }
        if (u.L > 0) {
            FirUpdate fu{};
            fu.flat = u.fir_dst;
            fu.L = u.L;
            fu.lpad = u.nkb * FIR_R;
            fu.taps = reinterpret_cast<float*>(p->dconst + u.off_taps);
            fu.plain = plain_at(pm, fu.flat);
            if (!fu.plain) return TFX_ERR_INVALID;
            f.push_back(fu);
        }
    }
    p->nsec = (int)v.size();
    p->nfir = (int)f.size();
    const size_t bytes = v.size() * sizeof(SecUpdate) + f.size() * sizeof(FirUpdate);
    if (bytes == 0) return TFX_OK;
    if (cudaMalloc(&p->dsec, bytes) != cudaSuccess) return TFX_ERR_NOMEM;
    if (!v.empty() && cudaMemcpy(p->dsec, v.data(), v.size() * sizeof(SecUpdate), cudaMemcpyHostToDevice) != cudaSuccess)
        return TFX_ERR_CUDA;
    if (!f.empty() && cudaMemcpy(p->dsec + v.size() * sizeof(SecUpdate), f.data(), f.size() * sizeof(FirUpdate),
                                 cudaMemcpyHostToDevice) != cudaSuccess)
        return TFX_ERR_CUDA;
    return TFX_OK;
}

// Coefficients derived on the host (the tensor-core cascade's GEMM tables,
// a composed chain's spectrum) go stale with an update: such units run the
// look-back scan, and the chain its separate units, from now on.  A spectral
// plan's chain spectrum is recomputed on the device instead.
void drop_host_derived(tfx_plan* p) {
    for (HostUnit& u : p->units) u.seg = false;
    if (!p->spectral) p->use_chain = false;
}

// A spectral plan after its sections (and FIR taps) changed: the FIR's
// spectrum at the chain's transform size from the new taps (coef, when
// given), the chain's spectrum from the new raw rows, and the decay check of
// the response against the overlap.
int refresh_spectral(tfx_plan* p, const double* coef, cudaStream_t s) {
    HostUnit& h = p->spec_fir;
    const float2* tw = reinterpret_cast<const float2*>(p->dconst + h.off_tw);
    float2* Hf = reinterpret_cast<float2*>(p->dconst + h.off_H);
    float2* H = reinterpret_cast<float2*>(p->dconst + p->chain.off_H);
    if (coef && p->spec_nfir &&
        launch_fir_fft_spectrum(coef + p->spec_fir_dst, h.L, h.fft_M, h.fft_B, 0, tw, Hf, s) != cudaSuccess)
        return TFX_ERR_CUDA;
    if (launch_chain_spectrum(reinterpret_cast<const double*>(p->dconst + p->off_spec_raw), p->chain_S, Hf,
                              reinterpret_cast<const double2*>(p->dconst + p->off_spec_z),
                              p->chain.fft_m, H, s) != cudaSuccess)
        return TFX_ERR_CUDA;
    if (launch_chain_tail(p->chain.fft_m, H, tw, p->chain.L - 1, p->dstatus, s) != cudaSuccess) return TFX_ERR_CUDA;
    return TFX_OK;
}

}  // namespace

int tfx::plan_update_sections(tfx_plan* p, const double* rows_dev, cudaStream_t s) {
    drop_host_derived(p);
    const int rc = build_update_descriptors(p);
    if (rc != TFX_OK) return rc;
    if (p->nsec <= 0) return TFX_OK;
    k_update_sections<<<(unsigned)p->nsec, 256, 0, s>>>(reinterpret_cast<const SecUpdate*>(p->dsec), rows_dev, 0,
                                                         p->dstatus);
    if (cudaGetLastError() != cudaSuccess) return TFX_ERR_CUDA;
    return p->spectral ? refresh_spectral(p, nullptr, s) : TFX_OK;
}

extern "C" int tfx_plan_update_sos(tfx_plan* p, const double* rows, tfx_stream s) {
    if (!p) return TFX_ERR_INVALID;
    int64_t nrows = 0;
    for (const HostUnit& u : p->units) nrows += u.S;
    if (nrows > 0 && !rows) return TFX_ERR_INVALID;
    return plan_update_sections(p, rows, reinterpret_cast<cudaStream_t>(s));
}

extern "C" int tfx_plan_update_coefs(tfx_plan* p, const double* coef, tfx_stream stream) {
    if (!p) return TFX_ERR_INVALID;
    if (p->ncoef > 0 && !coef) return TFX_ERR_INVALID;
    for (const HostUnit& u : p->units)
        if (u.tc) return TFX_ERR_UNSUPPORTED;  // tap tables scaled on the host
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    drop_host_derived(p);
    const int rc = build_update_descriptors(p);
    if (rc != TFX_OK) return rc;
    if (p->nsec > 0) {
        k_update_sections<<<(unsigned)p->nsec, 256, 0, s>>>(reinterpret_cast<const SecUpdate*>(p->dsec), coef, 1,
                                                             p->dstatus);
        if (cudaGetLastError() != cudaSuccess) return TFX_ERR_CUDA;
    }
    if (p->nfir > 0) {
        k_update_fir_taps<<<(unsigned)p->nfir, 256, 0, s>>>(
            reinterpret_cast<const FirUpdate*>(p->dsec + (size_t)p->nsec * sizeof(SecUpdate)), coef);
        if (cudaGetLastError() != cudaSuccess) return TFX_ERR_CUDA;
    }
    if (p->spectral) return refresh_spectral(p, coef, s);  // the units do not run
    for (const HostUnit& u : p->units) {
        if (!u.fft) continue;
        if (launch_fir_fft_spectrum(coef + u.fir_dst, u.L, u.fft_M, u.fft_B, u.fft_P,
                                    reinterpret_cast<const float2*>(p->dconst + u.off_tw),
                                    reinterpret_cast<float2*>(p->dconst + u.off_H), s) != cudaSuccess)
            return TFX_ERR_CUDA;
    }
    return TFX_OK;
}

extern "C" int tfx_plan_update_coefs_launch_count(const tfx_plan* p) {
    if (!p) return -1;
    int64_t S = 0;
    int n = 0;
    for (const HostUnit& u : p->units) {
        if (u.tc) return -1;
        S += u.S;
        if (u.fft) ++n;
    }
    bool fir = false;
    for (const HostUnit& u : p->units) fir = fir || u.L > 0;
    if (p->spectral) n = (p->spec_nfir ? 1 : 0) + 2;  // FIR spectrum, chain spectrum, decay check
    return (S > 0 ? 1 : 0) + (fir ? 1 : 0) + n;
}

extern "C" int64_t tfx_plan_sos_rows(const tfx_plan* p) {
    if (!p) return -1;
    int64_t n = 0;
    for (const HostUnit& u : p->units) n += u.S;
    return n;
}
