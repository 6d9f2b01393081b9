// Host side of libtfx: argument validation, plan building (FP64 precompute of
// device constants), workspace layout, launches, the one-shot plan cache and
// the C-ABI entry points declared in include/tfx.h.
#include <algorithm>
#include <cassert>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <list>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "plan_internal.cuh"

using namespace tfx;

// Tensor-core FIR geometry for L taps and NB output blocks per tile.
void tfx::tc_geometry(HostUnit& u, int NB) {
    u.W = ((u.L - 1 + 15) / 16) * 16;
    u.nK = (u.W + 128) / 16;
    u.NB = NB;
    u.rows = NB + (u.W + 127) / 128 + 1;
    u.tmem_cols = NB <= 32 ? 32 : (NB <= 64 ? 64 : (NB <= 128 ? 128 : 256));
    u.a_chunks = 2 * u.nK + 16;
    u.tc_smem = (size_t)u.a_chunks * 128 * 2 + (size_t)16 * u.rows * 16 * 2 + 16;
}


namespace {

// One step of a cascade's whole state in FP64 with input u: x = (w1_0, w2_0,
// ..., w1_(S-1), w2_(S-1)) -> x', each section driven by the previous one's
// output; returns the cascade output y = C x + D u.
double cascade_free_step(const std::vector<double>& sec, int S, const double* x, double* xn, double u) {
    double v = u;
    for (int i = 0; i < S; ++i) {
        const double* r = &sec[5 * (size_t)i];  // b0 b1 b2 a1 a2 (a0-normalised)
        const double c1 = r[1] - r[3] * r[0], c2 = r[2] - r[4] * r[0];
        const double w1 = x[2 * i], w2 = x[2 * i + 1];
        const double out = r[0] * v + w1;
        xn[2 * i] = c1 * v - r[3] * w1 + w2;
        xn[2 * i + 1] = c2 * v - r[4] * w1;
        v = out;
    }
    return v;
}

// 16 x 16 row-major products (state dimension 2S <= 16, zero-padded).
using Mat16 = std::array<double, 256>;
Mat16 mat_mul(const Mat16& a, const Mat16& b) {
    Mat16 c{};
    for (int r = 0; r < 16; ++r)
        for (int k = 0; k < 16; ++k) {
            const double ark = a[r * 16 + k];
            if (ark == 0.0) continue;
            for (int m = 0; m < 16; ++m) c[r * 16 + m] += ark * b[k * 16 + m];
        }
    return c;
}
Mat16 mat_eye() {
    Mat16 e{};
    for (int i = 0; i < 16; ++i) e[i * 17] = 1.0;
    return e;
}

uint16_t f2h(float f);  // FP32 -> FP16 bits and back, defined with the FIR tables below
double h2d(uint16_t h);

// Store v (row r, column k of a [rows x K] operand) into a canonical
// no-swizzle K-major FP16 table: (r % 8) * 16 + (r / 8) * SBO + (k % 8) * 2 +
// (k / 8) * 128 bytes.
void canon_put(uint8_t* base, int r, int k, int K, uint16_t v) {
    const size_t off = (size_t)(r % 8) * 16 + (size_t)(r / 8) * (K / 8) * 128 + (size_t)(k % 8) * 2 + (size_t)(k / 8) * 128;
    std::memcpy(base + off, &v, 2);
}

// Decide whether cascade unit u runs on the tensor cores by channel segments
// (k_sos_tc) and build its tables.  D: the free response y_n = C A^n s falls
// below 1e-9 of its initial size (the largest ||C A^n||_1 over n < 64) after
// n = D0 (the search stops once it has stayed below for D0 + 1024 steps, and
// gives up at 65536); D = 1.25 D0 rounded up to whole 112-sample blocks.
// Every segment but a channel's first runs D warm-up samples from zero state
// before its own range, so its state there is the true one to that accuracy.
// Segments: lengths a multiple of the 14336-sample tile and at least 4 D,
// their number P per channel minimising the per-SM work
// ceil(C P / SMs) x (tiles per segment + D / tile) (one persistent CTA per SM
// walks its segments).
void choose_segments(const tfx_plan* p, HostUnit& u, int sm_count) {
    const int S = u.S, n2 = 2 * S;
    Mat16 A{};
    std::vector<double> Crow(n2, 0.0);
    for (int m = 0; m < n2; ++m) {
        double x[16] = {0}, xn[16] = {0};
        x[m] = 1.0;
        Crow[m] = cascade_free_step(u.sec, S, x, xn, 0.0);
        for (int r = 0; r < n2; ++r) A[r * 16 + m] = xn[r];
    }
    std::vector<double> R = Crow, Rn(n2);
    double ref = 0.0;
    int64_t last = 0;
    bool decayed = false;
    for (int64_t n = 0; n < 65536; ++n) {
        double norm = 0.0;
        for (int r = 0; r < n2; ++r) norm += std::fabs(R[r]);
        if (n < 64) {
            ref = std::max(ref, norm);
        } else if (norm > 1e-9 * ref) {
            last = n;
        } else if (n > 2 * last + 1024) {
            decayed = true;
            break;
        }
        for (int m = 0; m < n2; ++m) {
            double acc = 0.0;
            for (int r = 0; r < n2; ++r) acc += R[r] * A[r * 16 + m];
            Rn[m] = acc;
        }
        R.swap(Rn);
    }
    if (!decayed) return;
    const int D = (int)(((int64_t)(1.25 * (double)(last + 1)) + TCS_KB - 1) / TCS_KB * TCS_KB);
    const int64_t tiles = (p->N + TCS_TILE - 1) / TCS_TILE;
    int64_t bestP = 1;
    double best = 0.0;
    for (int64_t P = 1; P <= tiles; ++P) {
        const int64_t tps = (tiles + P - 1) / P;  // tiles per segment
        if (P > 1 && tps * TCS_TILE < 4 * (int64_t)D) break;
        const double work = (double)((p->C * P + sm_count - 1) / sm_count) *
                            ((double)tps + (P > 1 ? (double)D / TCS_TILE : 0.0));
        if (P == 1 || work < best) bestP = P, best = work;
    }
    const int64_t tps = (tiles + bestP - 1) / bestP;
    const int64_t Lseg = tps * TCS_TILE;
    const int64_t P = (p->N + Lseg - 1) / Lseg;
    u.seg = true;
    u.seg_P = P;
    u.seg_len = Lseg;
    u.seg_D = P > 1 ? D : 0;

    // tensor-core tables.  Impulse response h, input-to-state columns
    // A^(111-k) B, free-response rows C A^m, block transfer A^112.
    double Bv[16] = {0}, x0[16] = {0};
    const double Dd = cascade_free_step(u.sec, S, x0, Bv, 1.0);
    std::vector<double> h(TCS_KB);
    h[0] = Dd;
    {
        double x[16], xn[16];
        std::copy(Bv, Bv + 16, x);
        for (int n = 1; n < TCS_KB; ++n) {
            double acc = 0.0;
            for (int r = 0; r < n2; ++r) acc += Crow[r] * x[r];
            h[n] = acc;
            for (int r = 0; r < 16; ++r) xn[r] = 0.0;
            for (int r = 0; r < n2; ++r)
                for (int m = 0; m < n2; ++m) xn[r] += A[r * 16 + m] * x[m];
            std::copy(xn, xn + 16, x);
        }
    }
    std::vector<double> A1((size_t)128 * TCS_KB, 0.0), A2((size_t)128 * 16, 0.0);
    for (int m = 0; m < TCS_KB; ++m)
        for (int k = 0; k <= m; ++k) A1[(size_t)m * TCS_KB + k] = h[m - k];
    {
        double col[16];
        std::copy(Bv, Bv + 16, col);  // A^0 B for k = 111
        for (int k = TCS_KB - 1; k >= 0; --k) {
            for (int r = 0; r < 16; ++r) A1[(size_t)(TCS_KB + r) * TCS_KB + k] = col[r];
            double nx[16] = {0};
            for (int r = 0; r < n2; ++r)
                for (int m = 0; m < n2; ++m) nx[r] += A[r * 16 + m] * col[m];
            std::copy(nx, nx + 16, col);
        }
        std::vector<double> row(Crow.begin(), Crow.end());
        row.resize(16, 0.0);
        for (int m = 0; m < TCS_KB; ++m) {
            for (int r = 0; r < 16; ++r) A2[(size_t)m * 16 + r] = row[r];
            double nr[16] = {0};
            for (int c = 0; c < n2; ++c)
                for (int r = 0; r < n2; ++r) nr[c] += row[r] * A[r * 16 + c];
            std::copy(nr, nr + 16, row.begin());
        }
    }
    u.tc_a1.assign((size_t)2 * TCS_A1_BYTES, 0);
    u.tc_a2.assign((size_t)2 * TCS_A2_BYTES, 0);
    u.tc_rowinv.assign(128, 1.f);
    for (int m = 0; m < 128; ++m) {
        double mx = 0.0;
        for (int k = 0; k < TCS_KB; ++k) mx = std::max(mx, std::fabs(A1[(size_t)m * TCS_KB + k]));
        for (int r = 0; r < 16; ++r) mx = std::max(mx, std::fabs(A2[(size_t)m * 16 + r]));
        int sh = 0;
        if (mx > 0.0) sh = std::max(-126, std::min(126, 14 - std::ilogb(mx)));
        const double sc = std::ldexp(1.0, sh);
        u.tc_rowinv[m] = (float)std::ldexp(1.0, -sh);
        for (int k = 0; k < TCS_KB; ++k) {
            const float v = (float)(A1[(size_t)m * TCS_KB + k] * sc);
            const uint16_t hi = f2h(v), lo = f2h((float)(v - h2d(hi)));
            canon_put(u.tc_a1.data(), m, k, TCS_KB, hi);
            canon_put(u.tc_a1.data() + TCS_A1_BYTES, m, k, TCS_KB, lo);
        }
        for (int r = 0; r < 16; ++r) {
            const float v = (float)(A2[(size_t)m * 16 + r] * sc);
            const uint16_t hi = f2h(v), lo = f2h((float)(v - h2d(hi)));
            canon_put(u.tc_a2.data(), m, r, 16, hi);
            canon_put(u.tc_a2.data() + TCS_A2_BYTES, m, r, 16, lo);
        }
    }
    Mat16 phib = mat_eye();
    for (int t = 0; t < TCS_KB; ++t) phib = mat_mul(phib, A);
    u.tc_phib.assign(8 * 256, 0.f);
    Mat16 phj = phib;
    for (int j = 0; j < 8; ++j) {
        for (int i = 0; i < 256; ++i) u.tc_phib[(size_t)j * 256 + i] = (float)phj[i];
        phj = mat_mul(phj, phib);
    }
}

// Overlap-save scheme for an L-tap FIR: transform size M = 2^m and number of
// partitions P (0: single-block, B = M - (L - 1) outputs per block; else
// partitions of B = M/2 taps).  The choice minimises a cost model fitted to
// measured GB300 times per output (16 channels x 2.88M samples, L2 flushed
// between calls, microseconds for the whole signal): single-block
// 30 + k_m M / B with k_m from FFT_K (the 30 is the memory traffic, the rest
// the transforms); partitioned I_m + s_m P with I = 219, 230, 253, 326, 357
// and s = 20, 21.4, 23.6, 24.7, 26 for m = 10..14 (two launches and the
// spectra traffic; m = 14 from the 16384-tap FIR, 2 partitions, 0.96 of the
// time of 8192 points with 4, its per-partition cost taken near m = 13's: the
// spectra bytes per output and partition do not depend on M).  A single
// block must hold B >= M/8 outputs.  `force` (10..14) restricts the choice
// to that m.
struct FftScheme {
    int M = 0, P = 0;
};

// Single-block cost per (M / B) for m = 10..14 (m = 14: one 512-thread CTA
// per SM, 32 points per thread), measured with B between M/4 and 7M/8.
const double FFT_K[5] = {60.0, 63.0, 72.0, 111.0, 125.0};

double fft_single_cost(int m, int L) {
    const int M = 1 << m, B = M - (L - 1);
    return B >= M / 8 ? 30.0 + FFT_K[m - 10] * M / B : -1.0;
}

FftScheme fft_scheme_for(int L, int force, double* cost_out = nullptr) {
    static const double I[5] = {219.0, 230.0, 253.0, 326.0, 357.0};
    static const double SP[5] = {20.0, 21.4, 23.6, 24.7, 26.0};
    FftScheme best;
    double cost = 0.0;
    for (int m = 10; m <= 14; ++m) {
        if (force >= 10 && force <= 14 && m != force) continue;
        const double c1 = fft_single_cost(m, L);
        if (c1 > 0.0 && (best.M == 0 || c1 < cost)) best.M = 1 << m, best.P = 0, cost = c1;
        if (m >= 11 || force == m) {
            const int M = 1 << m;
            const int P = (L + M / 2 - 1) / (M / 2);
            const double c = I[m - 10] + SP[m - 10] * P;
            if (best.M == 0 || c < cost) best.M = M, best.P = P, cost = c;
        }
    }
    if (cost_out) *cost_out = cost;
    return best;
}

// In-place iterative radix-2 FFT (FP64), natural order in and out.
void host_fft(std::vector<std::complex<double>>& a) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

// Linear convolution a * b by FP64 transforms (zero-padded to a power of
// two), its first nout values.
std::vector<double> conv_fft(const std::vector<double>& a, const std::vector<double>& b, size_t nout) {
    const size_t need = a.size() + b.size() - 1;
    size_t n = 1;
    while (n < need) n <<= 1;
    std::vector<std::complex<double>> fa(n, 0.0), fb(n, 0.0);
    for (size_t i = 0; i < a.size(); ++i) fa[i] = a[i];
    for (size_t i = 0; i < b.size(); ++i) fb[i] = b[i];
    host_fft(fa);
    host_fft(fb);
    for (size_t i = 0; i < n; ++i) fa[i] = std::conj(fa[i] * fb[i]);
    host_fft(fa);  // conj(FFT(conj(X))) / n is the inverse
    std::vector<double> out(std::min(nout, need));
    for (size_t i = 0; i < out.size(); ++i) out[i] = fa[i].real() / (double)n;
    return out;
}

// Twiddle tables of the overlap-save transform of M = 2^m points: its passes
// run over spans M, M/G0, ..., 16 (G0 = 2^(m mod 4), or 16), radix G0 first
// and 16 after (32 points per thread, m = 14: spans M, M/32, 16 with radix
// 32, 32, 16); a pass over span S with radix G and sub = S/G > 1 has the
// twiddles w(q, i) = e^(-2 pi i * i * bitrev_G(q) / S), q = 1..G-1, i < sub,
// stored as pairs (w(2k + 1, i), w(2k + 2, i)) at [k][i], then the row of
// w(G - 1, i) when G - 1 is odd.
std::vector<std::complex<double>> fft_pass_twiddles(int m) {
    std::vector<std::complex<double>> out;
    const int M = 1 << m, r = m % 4;
    std::vector<std::pair<int, int>> passes;
    int S = M;
    if (fft_pt(m) == 32) {
        for (; S > 16; S >>= 5) passes.push_back({S, 32});
        passes.push_back({16, 16});
    } else {
        if (r) {
            passes.push_back({S, 1 << r});
            S >>= r;
        }
        for (; S >= 16; S >>= 4) passes.push_back({S, 16});
    }
    for (const auto& ps : passes) {
        const int Sp = ps.first, G = ps.second, sub = Sp / G;
        if (sub == 1) continue;
        int bits = 0;
        while ((1 << bits) < G) ++bits;
        auto tw = [&](int q, int i) {
            int kq = 0;
            for (int b = 0; b < bits; ++b) kq |= ((q >> b) & 1) << (bits - 1 - b);
            const double ang = -2.0 * M_PI * (double)(((int64_t)i * kq) % Sp) / (double)Sp;
            return std::complex<double>(std::cos(ang), std::sin(ang));
        };
        // slots 2k + 1 and 2k + 2 interleaved per group position, then the
        // last slot of an odd count alone
        for (int q = 1; q + 1 < G; q += 2)
            for (int i = 0; i < sub; ++i) {
                out.push_back(tw(q, i));
                out.push_back(tw(q + 1, i));
            }
        if ((G - 1) % 2 == 1)
            for (int i = 0; i < sub; ++i) out.push_back(tw(G - 1, i));
    }
    return out;
}

}  // namespace

namespace {

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Normalise one row by a0 and check that both poles lie strictly inside the
// unit circle: z^2 + al1 z + al2 has its roots in |z| < 1 iff |al2| < 1 and
// |al1| < 1 + al2.
int normalise_row(const double* r, double* out) {
    if (r[3] == 0.0) return TFX_ERR_INVALID;
    const double inv = 1.0 / r[3];
    const double b0 = r[0] * inv, b1 = r[1] * inv, b2 = r[2] * inv, al1 = r[4] * inv, al2 = r[5] * inv;
    if (!(std::fabs(al2) < 1.0 && std::fabs(al1) < 1.0 + al2)) return TFX_ERR_UNSTABLE;
    out[0] = b0;
    out[1] = b1;
    out[2] = b2;
    out[3] = al1;
    out[4] = al2;
    return TFX_OK;
}

// Device coefficients of one a0-normalised section (b0 b1 b2 a1 a2): the
// recursion w1' = c1 u - a1 w1 + w2, w2' = c2 u - a2 w1, y = b0 u + w1 uses
// c1 = b1 - a1 b0 and c2 = b2 - a2 b0, formed here in FP64 before rounding.
// Slot 5 holds d = a1 b2 - a2 b1, which maps the adjoint all-pole state to the
// state of the section run backwards in time (used by the backward kernel).
void sec_device_coefs(const double* r, float* out) {
    out[0] = (float)r[0];
    out[1] = (float)(r[1] - r[3] * r[0]);
    out[2] = (float)(r[2] - r[4] * r[0]);
    out[3] = (float)r[3];
    out[4] = (float)r[4];
    out[5] = (float)(r[3] * r[2] - r[4] * r[1]);
}

// Round-to-nearest-even FP32 -> BF16 bits, and back.
uint16_t f2bf(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
// Round-to-nearest-even FP32 -> IEEE FP16 bits (subnormals included), and back.
uint16_t f2h(float f) {
    uint32_t x;
    std::memcpy(&x, &f, 4);
    const uint32_t sign = (x >> 16) & 0x8000u;
    const uint32_t mant = x & 0x7fffffu;
    const int exp = (int)((x >> 23) & 0xffu);
    if (exp == 0xff) return (uint16_t)(sign | 0x7c00u | (mant ? 0x200u : 0u));
    const int e = exp - 127;
    if (e > 15) return (uint16_t)(sign | 0x7c00u);
    if (e >= -14) {
        uint32_t h = ((uint32_t)(e + 15) << 10) | (mant >> 13);
        const uint32_t rem = mant & 0x1fffu;
        if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) h += 1u;
        return (uint16_t)(sign | h);
    }
    if (e < -25 || exp == 0) return (uint16_t)sign;
    const uint32_t m = mant | 0x800000u;
    const int shift = -e - 1;
    uint32_t r = m >> shift;
    const uint32_t rem = m & ((1u << shift) - 1u), half = 1u << (shift - 1);
    if (rem > half || (rem == half && (r & 1u))) r += 1u;
    return (uint16_t)(sign | r);
}
double h2d(uint16_t h) {
    const int e = (h >> 10) & 0x1f, m = h & 0x3ff;
    const double v = e == 0 ? std::ldexp((double)m, -24) : std::ldexp(1.0 + m / 1024.0, e - 15);
    return (h & 0x8000u) ? -v : v;
}
float bf2f(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Pick the tile width for a tensor-core FIR: 128 blocks (16384 outputs) when
// two CTAs fit on an SM, else the widest that fits one CTA; false if none does.
bool choose_tc(HostUnit& u) {
    // persistent kernel: NB = 128, two window stages next to the resident taps
    tc_geometry(u, 128);
    u.tc_smem_ws = (size_t)u.a_chunks * 128 * 2 + (size_t)16 * u.rows * 16 * 4 + 10 * 8 + 12 * 4 + 32;
    if (u.tc_smem_ws <= SMEM_MAX) {
        u.tc_variant = 1;
        return true;
    }
    // long FIRs: taps streamed in K-blocks, one resident window
    u.tc_smem_ws = fir_tc_long_smem(u.rows);
    if (u.tc_smem_ws <= SMEM_MAX) {
        u.tc_variant = 2;
        return true;
    }
    const int cands[] = {128, 256, 64};
    for (int nb : cands) {
        tc_geometry(u, nb);
        if (nb == 128 && u.tc_smem <= 110 * 1024) return true;
        if (nb != 128 && u.tc_smem <= SMEM_MAX) return true;
    }
    tc_geometry(u, 128);
    return u.tc_smem <= SMEM_MAX;
}

struct M2 {
    double a, b, c, d;
};
inline M2 mul(const M2& x, const M2& y) {
    return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}

int validate_stages(const tfx_stage* st, int32_t nst) {
    if (nst < 0 || (nst > 0 && !st)) return TFX_ERR_INVALID;
    for (int32_t i = 0; i < nst; ++i) {
        const tfx_stage& s = st[i];
        if (s.kind == TFX_STAGE_FIR) {
            if (s.n < 1 || !s.coef || !finite_all(s.coef, (size_t)s.n)) return TFX_ERR_INVALID;
        } else if (s.kind == TFX_STAGE_SOS) {
            if (s.n < 0 || (s.n > 0 && !s.coef)) return TFX_ERR_INVALID;
            if (s.n > 0 && !finite_all(s.coef, (size_t)s.n * 6)) return TFX_ERR_INVALID;
            double tmp[5];
            for (int r = 0; r < s.n; ++r) {
                int e = normalise_row(s.coef + 6 * r, tmp);
                if (e != TFX_OK) return e;
            }
        } else {
            return TFX_ERR_INVALID;
        }
    }
    return TFX_OK;
}

int check_dims(int64_t C, int64_t N, int64_t ld) {
    if (C < 0 || N < 0) return TFX_ERR_INVALID;
    if (ld < (N > 1 ? N : 1)) return TFX_ERR_INVALID;
    if (C > 0 && N > 0) {
        // tile counts and indices stay within 32-bit grid / ticket ranges
        const int64_t ntt = (N + TILE - 1) / TILE;
        if (C > (int64_t)INT32_MAX / ntt) return TFX_ERR_UNSUPPORTED;
        if (C > INT64_MAX / ld) return TFX_ERR_INVALID;
    }
    return TFX_OK;
}

// Estimated time of a unit on 16 channels x 2.88M samples (microseconds, the
// scale of the FFT cost model), to compare a composed chain with its units.
double unit_cost_estimate(const HostUnit& u) {
    if (u.fft) {
        double c = 0.0;
        const FftScheme sch = fft_scheme_for(u.L, u.fft_P > 0 ? 0 : u.fft_m, &c);
        return sch.M > 0 ? c : 200.0;
    }
    if (u.tc) return 60.0 + 0.15 * u.L;  // persistent tensor-core GEMM, ~209 us at 1025 taps
    if (u.seg) return 140.0;             // tensor-core cascade by segments (8 sections, 16 x 2.88M: ~140 us)
    if (u.S > 0) return 220.0 + (u.L > 0 ? 2.0 * u.L : 0.0);  // look-back scan (+ fused CUDA-core FIR)
    return 40.0 + 2.0 * u.L;             // CUDA-core FIR
}

// Truncation threshold of the composite response, relative to the chain's
// RMS gain: at this level the dropped tail is no larger than the FP32
// transform's own rounding of the outputs (a few 1e-7 of the output peak).
constexpr double COMPOSE_EPS = 1e-7;

// The cascades' impulse response g (sections [S][5] in chain order, FP64,
// zero state) over 65536 samples and the length D it is truncated to when it
// is convolved with the FIR taps f: the first D for which
// sum_(n >= D) |g[n]| * sum |f| <= 1e-7 ||g * f||_2 (COMPOSE_EPS).  False when g has not
// decayed by the end (the absolute sum of its last 4096 samples above 1e-14
// of the whole) or the chain's response is zero.
bool cascade_decay(const std::vector<double>& sec, int S, const std::vector<double>& f, std::vector<double>& g,
                   int& D) {
    const int W = 65536, HEAD = 16384;
    g.assign(W, 0.0);
    std::vector<double> w1(S, 0.0), w2(S, 0.0);
    for (int n = 0; n < W; ++n) {
        double v = n == 0 ? 1.0 : 0.0;
        for (int i = 0; i < S; ++i) {
            const double* r = &sec[5 * (size_t)i];  // b0 b1 b2 a1 a2
            const double c1 = r[1] - r[3] * r[0], c2 = r[2] - r[4] * r[0];
            const double out = r[0] * v + w1[i];
            const double n1 = c1 * v - r[3] * w1[i] + w2[i];
            w2[i] = c2 * v - r[4] * w1[i];
            w1[i] = n1;
            v = out;
        }
        g[n] = v;
    }
    double total = 0.0, last = 0.0;
    for (int n = 0; n < W; ++n) total += std::fabs(g[n]);
    for (int n = W - 4096; n < W; ++n) last += std::fabs(g[n]);
    if (!(total > 0.0) || !(last <= 1e-14 * total)) return false;
    double f1 = 0.0, n2 = 0.0;
    for (double v : f) f1 += std::fabs(v);
    {
        const std::vector<double> head(g.begin(), g.begin() + HEAD);
        for (double v : conv_fft(head, f, HEAD)) n2 += v * v;
        n2 = std::sqrt(n2);
    }
    if (!(n2 > 0.0)) return false;
    D = W;
    double tail = 0.0;
    for (int n = W - 1; n >= 1; --n) {
        if ((tail + std::fabs(g[n])) * f1 > COMPOSE_EPS * n2) {
            D = n + 1;
            break;
        }
        tail += std::fabs(g[n]);
        D = n;
    }
    return true;
}

// The whole chain as one FIR (the pipe composes linear time-invariant stages,
// so the chain is the convolution with its composite impulse response).  The
// cascades' impulse response g (all sections in chain order, FP64, zero
// state) is computed over 65536 samples and must have decayed there (the
// absolute sum of its last 4096 samples below 1e-14 of the whole).  With f
// every FIR's taps convolved (FP64), g is truncated at the first D for which
// sum_(n >= D) |g[n]| * sum |f| <= 1e-7 ||h_c||_2: the truncated tail changes
// no output by more than that times max|x|, and ||h_c||_2 is the chain's RMS
// gain for white input (taken over the first 16384 samples of h_c = g * f, a
// lower bound).  The composite h_c = g[0, D) * f has Lc = D + Lf - 1 taps and
// runs by single-block overlap-save with the transform size of least
// modelled cost, if that beats the separate units (a chain of cascades alone
// too: f is then the unit impulse); the signal must hold at
// least 2 Lc samples (the transform's rounding is relative to each block's
// energy, so a signal shorter than the response would be compared with an
// output made only of its smallest leading terms).
void compose_chain(tfx_plan* p) {
    int S = 0;
    std::vector<double> sec;
    std::vector<double> f(1, 1.0);
    int maxL = 0;
    double separate = 0.0;
    for (const HostUnit& u : p->units) {
        if (u.hiq) return;
        sec.insert(sec.end(), u.sec.begin(), u.sec.end());
        S += u.S;
        if (u.L > 0) {
            f = conv_fft(f, u.taps, f.size() + u.taps.size() - 1);
            maxL = std::max(maxL, u.L);
        }
        // a cascade-only unit of <= 8 sections would run on the tensor cores by segments
        HostUnit e = u;
        e.seg = u.S > 0 && u.S <= SEG_SMAX && u.L == 0 && !u.warp;
        separate += unit_cost_estimate(e);
    }
    if (S == 0) return;  // no cascade: a lone FIR is already one FFT FIR
    std::vector<double> g;
    int D = 0;
    if (!cascade_decay(sec, S, f, g, D)) return;
    const int Lf = (int)f.size();
    const int64_t Lc = (int64_t)D + Lf - 1;
    if (p->N < 2 * Lc) return;
    int bestm = 0;
    double best = 0.0;
    for (int m = 10; m <= 14; ++m) {
        const int M = 1 << m;
        if (Lc - 1 > M - M / 4) continue;  // at least M/4 outputs per block
        const double c = fft_single_cost(m, (int)Lc);
        if (c > 0.0 && (bestm == 0 || c < best)) bestm = m, best = c;
    }
    // a transform size set for this length bucket (the batch autotuner's
    // choice) where it holds the response with M/4 outputs per block
    int lg = 0;
    while (lg < 15 && (int64_t(2) << lg) <= Lc) ++lg;
    const int om = p->compose_m[lg];
    if (om >= 10 && om <= 14 && Lc - 1 <= (1 << om) - (1 << om) / 4) {
        bestm = om;
    } else if (bestm == 0 || !(best < separate)) {
        return;
    }
    HostUnit c;
    c.L = (int)Lc;
    c.taps = conv_fft(std::vector<double>(g.begin(), g.begin() + D), f, (size_t)Lc);
    c.fft = true;
    c.fft_m = bestm;
    c.fft_M = 1 << bestm;
    c.fft_P = 0;
    c.fft_B = c.fft_M - (c.L - 1);
    p->chain = c;
    p->use_chain = true;
    p->chain_S = S;
    p->chain_L = Lf;
    p->chain_D = D;
}

// A trainable chain whose stages all compose (cascades of at most SPEC_SMAX
// sections together, none with a pole above HIQ_RADIUS, and at most one FIR)
// trains by its composite spectrum.  The forward and the input gradient are
// single-block overlap-save FFT FIRs whose spectrum is the chain's transfer
// function evaluated in closed form at the transform's bins (the DFT of the
// untruncated response aliased M-periodically), and the coefficient
// gradients are inner products of the derivative spectra with the
// accumulated gradient-input cross-spectrum (k_spectral.cu).  The overlap J
// covers 1.5 D + Lf - 1 lags (D the decay length of cascade_decay; the
// margin holds the slower n r^n decay of the derivative responses and pole
// movement during training, and a device check after every coefficient
// update reports a response that outgrows it), at least M/4, with the
// smaller of 4096 and 8192 points that leaves M/4 outputs per block.  The
// signal must hold 2 (J + 1) samples (as for a composed chain).
void choose_spectral(tfx_plan* p) {
    int S = 0, nfir = 0;
    std::vector<double> sec, f(1, 1.0);
    int64_t fir_dst = 0;
    for (const HostUnit& u : p->units) {
        if (u.hiq) return;
        sec.insert(sec.end(), u.sec.begin(), u.sec.end());
        S += u.S;
        if (u.L > 0) {
            ++nfir;
            f = u.taps;
            fir_dst = u.fir_dst;
        }
    }
    if (S < 1 || S > SPEC_SMAX || nfir > 1) return;
    std::vector<double> g;
    int D = 0;
    if (!cascade_decay(sec, S, f, g, D)) return;
    const int Lf = (int)f.size();
    const int64_t Jn = (3 * (int64_t)D + 1) / 2 + Lf - 1;
    int m = 0;
    for (int mm = 12; mm <= 13 && m == 0; ++mm)
        if (Jn <= 3 * (int64_t(1) << mm) / 4) m = mm;
    if (m == 0) return;
    const int M = 1 << m;
    const int J = (int)std::max<int64_t>(Jn, M / 4);
    if (p->N < 2 * ((int64_t)J + 1)) return;
    HostUnit h;
    h.L = Lf;
    h.taps = f;
    h.fft = true;
    h.fft_m = m;
    h.fft_M = M;
    h.fft_P = 0;
    h.fft_B = M - (Lf - 1);
    HostUnit c;
    c.L = J + 1;
    c.fft = true;
    c.fft_m = m;
    c.fft_M = M;
    c.fft_P = 0;
    c.fft_B = M - J;
    p->spec_fir = h;
    p->spec_nfir = nfir;
    p->spec_fir_dst = fir_dst;
    p->chain = c;
    p->use_chain = true;
    p->spectral = true;
    p->chain_S = S;
    p->chain_L = nfir ? Lf : 0;
    p->chain_D = D;
}

// Spectrum of an FFT unit's taps (or of each partition) and its pass
// twiddles into the constant blob at the unit's offsets.
void fill_fft_tables(const HostUnit& u, char* host) {
    // spectrum of h zero-padded to M, scaled by 1/M (the inverse FFT's
    // normalisation), in bit-reversed order; twiddles e^(-2 pi i k / M)
    // (partitioned: of each partition h[pB, (p + 1) B))
    const int M = u.fft_M;
    const int parts = std::max(u.fft_P, 1), plen = u.fft_P > 0 ? u.fft_B : u.L;
    for (int q = 0; q < parts; ++q) {
        std::vector<std::complex<double>> Hc(M, 0.0);
        for (int k = 0; k < plen && q * plen + k < u.L; ++k) Hc[k] = u.taps[q * plen + k];
        host_fft(Hc);
        // position k = PT t + 2c + e (thread t, float4 c, half e; PT points
        // per thread) holds H[bitrev(k)] / M and is stored at float2 index
        // 2 (c T + t) + e
        float2* Hd = reinterpret_cast<float2*>(host + u.off_H) + (size_t)q * M;
        const int PT = fft_pt(u.fft_m), T = M / PT;
        for (int k = 0; k < M; ++k) {
            int r = 0;
            for (int b = 0; b < u.fft_m; ++b) r |= ((k >> b) & 1) << (u.fft_m - 1 - b);
            const int t = k / PT, c = (k % PT) / 2, e = k % 2;
            Hd[2 * (c * T + t) + e] = make_float2((float)(Hc[r].real() / M), (float)(Hc[r].imag() / M));
        }
    }
    const std::vector<std::complex<double>> twd = fft_pass_twiddles(u.fft_m);
    float2* tw = reinterpret_cast<float2*>(host + u.off_tw);
    for (size_t k = 0; k < twd.size(); ++k) tw[k] = make_float2((float)twd[k].real(), (float)twd[k].imag());
}

int build_plan(tfx_plan* p, const tfx_stage* st, int32_t nst, bool upload) {
    // group stages: consecutive SOS stages merge into one cascade; an FIR
    // closes the current unit.
    HostUnit cur;
    auto flush = [&]() {
        if (cur.S > 0 || cur.L > 0) p->units.push_back(cur);
        cur = HostUnit();
    };
    // A trainable plan keeps every FIR in a unit of its own and at most
    // BWD_SMAX sections per cascade, and records where each coefficient's
    // gradient goes (stages in order; FIR: n taps, SOS: 6 values per row).
    p->train = (p->flags & TFX_PLAN_TRAINABLE) != 0;
    const bool unfused = (p->flags & TFX_PLAN_UNFUSED) != 0 || p->train;
    int64_t coff = 0;
    for (int32_t i = 0; i < nst; ++i) {
        const tfx_stage& s = st[i];
        if (s.kind == TFX_STAGE_SOS) {
            if (cur.L > 0) flush();
            for (int r = 0; r < s.n; ++r) {
                if (p->train && cur.S == BWD_SMAX) flush();
                double row[5];
                normalise_row(s.coef + 6 * r, row);
                cur.sec.insert(cur.sec.end(), row, row + 5);
                cur.S++;
                cur.dst.push_back(coff + 6 * r);
                cur.raw.insert(cur.raw.end(), s.coef + 6 * r, s.coef + 6 * r + 6);
            }
            coff += 6 * (int64_t)s.n;
        } else {
            if (unfused && cur.S > 0) flush();
            if (cur.L > 0) flush();
            cur.L = s.n;
            cur.taps.assign(s.coef, s.coef + s.n);
            cur.fir_dst = coff;
            cur.Lp = (s.n + 15) / 16 * 16;
            coff += s.n;
            flush();
        }
    }
    flush();
    p->ncoef = coff;

    // cascades with a pole of radius > HIQ_RADIUS run the warp-tile scan with
    // FP64 cross-tile carries; a short FIR fused behind one becomes its own unit
    if (p->allow_hiq) {
        std::vector<HostUnit> out;
        for (HostUnit& u : p->units) {
            for (int s = 0; s < u.S; ++s) {
                const double a1 = u.sec[5 * s + 3], a2 = u.sec[5 * s + 4];
                const double disc = a1 * a1 - 4.0 * a2;
                const double r = disc < 0.0 ? std::sqrt(a2)
                                            : std::max(std::fabs(-a1 + std::sqrt(disc)), std::fabs(-a1 - std::sqrt(disc))) / 2.0;
                if (r > HIQ_RADIUS) u.hiq = true;
            }
            if (u.hiq && u.L > 0) {
                HostUnit sos = u, fir = u;
                sos.L = 0;
                sos.taps.clear();
                fir.S = 0;
                fir.sec.clear();
                fir.hiq = false;
                fir.dst.clear();
                fir.raw.clear();
                out.push_back(sos);
                out.push_back(fir);
            } else {
                out.push_back(u);
            }
        }
        p->units.swap(out);
    }

    // long FIRs go to the tensor cores; an SOS cascade in front of one runs as
    // its own unit (the cascade output crosses HBM once more)
    if (!(p->flags & TFX_PLAN_FIR_CUDA_CORES)) {
        std::vector<HostUnit> out;
        for (HostUnit& u : p->units) {
            HostUnit f = u;
            // FFT overlap-save: forced for 64 taps or more, by default from
            // FFT_MIN_TAPS on unless a tensor-core mode or precision is asked for
            const int force = (int)((p->flags & TFX_PLAN_FIR_FFT_LOG_MASK) >> 16);
            const bool tc_only = (p->flags & (TFX_PLAN_FIR_TC | TFX_PLAN_FIR_BF16_PLAIN | TFX_PLAN_FIR_BF16_SPLIT)) != 0;
            // (by default only for signals of at least 2L samples: the
            // transform rounds relative to each block's energy, and a signal
            // shorter than the taps is all leading transient)
            const bool want_fft = (p->flags & TFX_PLAN_FIR_FFT)
                                      ? u.L >= 64
                                      : (!tc_only && u.L >= FFT_MIN_TAPS && p->N >= 2 * (int64_t)u.L);
            const FftScheme sch = want_fft ? fft_scheme_for(u.L, force) : FftScheme();
            const int fftM = sch.M, fftP = sch.P;
            if (fftM > 0) {
                f.S = 0;
                f.sec.clear();
                f.hiq = false;
                f.dst.clear();
                f.raw.clear();
                f.fft = true;
                f.fft_M = fftM;
                f.fft_m = 0;
                while ((1 << f.fft_m) < fftM) ++f.fft_m;
                f.fft_P = fftP;
                f.fft_B = fftP > 0 ? fftM / 2 : fftM - (u.L - 1);
                if (u.S > 0) {
                    HostUnit sos = u;
                    sos.L = 0;
                    sos.taps.clear();
                    out.push_back(sos);
                }
                out.push_back(f);
            } else if (u.L >= p->tc_min_taps && (f.S = 0, f.sec.clear(), choose_tc(f))) {
                f.tc = true;
                if (u.S > 0) {
                    HostUnit sos = u;
                    sos.L = 0;
                    sos.taps.clear();
                    out.push_back(sos);
                }
                out.push_back(f);
            } else {
                out.push_back(u);
            }
        }
        p->units.swap(out);
    }

    for (HostUnit& u : p->units)
        u.warp = (u.S > 0 && u.L == 0) && ((p->flags & TFX_PLAN_SCAN_WARP_TILES) || p->train || u.hiq);

    // the whole chain as one FFT FIR of its composite response
    p->use_chain = false;
    if (!(p->flags & (TFX_PLAN_NO_COMPOSE | TFX_PLAN_FIR_CUDA_CORES | TFX_PLAN_UNFUSED | TFX_PLAN_FIR_BF16_PLAIN |
                      TFX_PLAN_FIR_BF16_SPLIT | TFX_PLAN_SCAN_WARP_TILES | TFX_PLAN_FIR_TC | TFX_PLAN_SCAN_LOOKBACK |
                      TFX_PLAN_TEST_DROP_PUBLISH | TFX_PLAN_FIR_FFT_LOG_MASK)) &&
        p->C > 0 && p->N > 0) {
        if (!p->train)
            compose_chain(p);
        else
            choose_spectral(p);
    }

    // cascade-only block-tile units by channel segments where the free
    // response decays early enough (not needed when the chain is composed:
    // after a coefficient update its units run the look-back scan)
    if (!(p->flags & (TFX_PLAN_SCAN_LOOKBACK | TFX_PLAN_TEST_DROP_PUBLISH)) && p->C > 0 && p->N > 0 && !p->use_chain) {
        int sm_count = 152, dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
        for (HostUnit& u : p->units)
            if (u.S > 0 && u.S <= SEG_SMAX && u.L == 0 && !u.warp && !u.hiq) {
                assert(!p->train);  // launch_unit_range's training callers pass no copy buffer
                choose_segments(p, u, sm_count);
            }
    }

    // constant blob layout (a spectral plan: every section's raw row and
    // gradient slot first, contiguous over the units)
    size_t off = 0;
    size_t spec_rows = 0;
    if (p->spectral) {
        p->off_spec_raw = off;
        off = align_up(off + (size_t)p->chain_S * 6 * sizeof(double));
        p->off_spec_dst = off;
        off = align_up(off + (size_t)p->chain_S * sizeof(int64_t));
    }
    for (HostUnit& u : p->units) {
        u.off_coef = off;
        off = align_up(off + (size_t)u.S * 8 * sizeof(float));
        u.off_pw = off;
        off = align_up(off + (size_t)u.S * PW_LEN * sizeof(float4));
        if (u.hiq) {
            u.off_pw64 = off;
            off = align_up(off + (size_t)u.S * PW_LEN * sizeof(double4));
        }
        u.nkb = u.L > 0 ? (u.L + FIR_R - 1) / FIR_R : 0;
        u.off_taps = off;
        off = align_up(off + (size_t)u.nkb * FIR_R * sizeof(float));
        if (u.tc) {
            u.off_ahi = off;
            off = align_up(off + (size_t)u.a_chunks * 128);
            u.off_alo = off;
            off = align_up(off + (size_t)u.a_chunks * 128);
        }
        if (u.seg) {
            u.off_tc = off;
            off = align_up(off + u.tc_a1.size() + u.tc_a2.size() + (u.tc_rowinv.size() + u.tc_phib.size()) * 4);
        }
        if (u.fft) {
            u.off_H = off;
            off = align_up(off + (size_t)std::max(u.fft_P, 1) * u.fft_M * sizeof(float2));
            u.off_tw = off;
            off = align_up(off + fft_pass_twiddles(u.fft_m).size() * sizeof(float2));
        }
        if (p->train && u.S > 0 && p->spectral) {
            u.off_raw = p->off_spec_raw + spec_rows * 6 * sizeof(double);
            u.off_dst = p->off_spec_dst + spec_rows * sizeof(int64_t);
            spec_rows += (size_t)u.S;
        } else if (p->train && u.S > 0) {
            u.off_raw = off;
            off = align_up(off + (size_t)u.S * 6 * sizeof(double));
            u.off_dst = off;
            off = align_up(off + (size_t)u.S * sizeof(int64_t));
        }
    }
    if (p->spectral) {  // the bins' z, the FIR's spectrum Hf and the twiddles (shared with the chain)
        p->off_spec_z = off;
        off = align_up(off + (size_t)p->spec_fir.fft_M * sizeof(double2));
        p->spec_fir.off_H = off;
        off = align_up(off + (size_t)p->spec_fir.fft_M * sizeof(float2));
        p->spec_fir.off_tw = off;
        off = align_up(off + fft_pass_twiddles(p->spec_fir.fft_m).size() * sizeof(float2));
        p->chain.off_tw = p->spec_fir.off_tw;
    }
    if (p->use_chain) {
        p->chain.off_H = off;
        off = align_up(off + (size_t)p->chain.fft_M * sizeof(float2));
        if (!p->spectral) {
            p->chain.off_tw = off;
            off = align_up(off + fft_pass_twiddles(p->chain.fft_m).size() * sizeof(float2));
        }
    }
    for (int32_t i = 0; i < nst; ++i) {
        PlainStage ps{st[i].kind, st[i].n, off};
        p->plain.push_back(ps);
        off = align_up(off + (size_t)(st[i].kind == TFX_STAGE_SOS ? st[i].n * 8 : st[i].n) * sizeof(float));
    }
    const size_t const_bytes = off;

    std::vector<char> host(const_bytes > 0 ? const_bytes : 1, 0);
    for (HostUnit& u : p->units) {
        float* coef = reinterpret_cast<float*>(host.data() + u.off_coef);
        float4* pw = reinterpret_cast<float4*>(host.data() + u.off_pw);
        for (int s = 0; s < u.S; ++s) {
            const double* r = &u.sec[5 * s];
            sec_device_coefs(r, coef + 8 * s);
            // one-sample transfer of the TDF-II state (w1, w2) with zero input
            const M2 m = {-r[3], 1.0, -r[4], 0.0};
            M2 a = {1, 0, 0, 1};
            const int chunk = u.L == 0 && !u.warp ? T_CASCADE : T_CHUNK;  // samples per thread of u's kernel
            for (int t = 0; t < chunk; ++t) a = mul(a, m);                 // chunk transfer A = M^chunk
            M2 pk = {1, 0, 0, 1};
            double4* pw64 = u.hiq ? reinterpret_cast<double4*>(host.data() + u.off_pw64) : nullptr;
            for (int k = 0; k < PW_LEN; ++k) {
                pw[(size_t)s * PW_LEN + k] = make_float4((float)pk.a, (float)pk.b, (float)pk.c, (float)pk.d);
                if (pw64) pw64[(size_t)s * PW_LEN + k] = make_double4(pk.a, pk.b, pk.c, pk.d);
                pk = mul(pk, a);
            }
        }
        float* taps = reinterpret_cast<float*>(host.data() + u.off_taps);
        for (int k = 0; k < u.L; ++k) taps[k] = (float)u.taps[k];
        if (u.seg) {
            char* t = host.data() + u.off_tc;
            std::memcpy(t, u.tc_a1.data(), u.tc_a1.size());
            std::memcpy(t + u.tc_a1.size(), u.tc_a2.data(), u.tc_a2.size());
            std::memcpy(t + u.tc_a1.size() + u.tc_a2.size(), u.tc_rowinv.data(), u.tc_rowinv.size() * 4);
            std::memcpy(t + u.tc_a1.size() + u.tc_a2.size() + u.tc_rowinv.size() * 4, u.tc_phib.data(),
                        u.tc_phib.size() * 4);
        }
        if (u.fft) fill_fft_tables(u, host.data());
        if (p->train && u.S > 0) {
            std::memcpy(host.data() + u.off_raw, u.raw.data(), (size_t)u.S * 6 * sizeof(double));
            std::memcpy(host.data() + u.off_dst, u.dst.data(), (size_t)u.S * sizeof(int64_t));
        }
        if (u.tc) {
            // g[v] = h[W + 127 - v]; chunk j, copy b holds g[8j + b .. 8j + b + 7].
            // FP16 mode: taps scaled by 2^e so that max|h| lands in [2^14, 2^15).
            u.tc_mode = (p->flags & TFX_PLAN_FIR_BF16_PLAIN) ? FIR_TC_BF16_PLAIN
                        : (p->flags & TFX_PLAN_FIR_BF16_SPLIT) ? FIR_TC_BF16_SPLIT : FIR_TC_FP16_SPLIT;
            double hmax = 0.0;
            for (double v : u.taps) hmax = std::max(hmax, std::fabs(v));
            int sh = 0;
            if (u.tc_mode == FIR_TC_FP16_SPLIT && hmax > 0.0) {
                sh = 14 - std::ilogb(hmax);
                sh = sh > 126 ? 126 : (sh < -126 ? -126 : sh);
            }
            u.tap_unscale = (float)std::ldexp(1.0, -sh);
            uint16_t* hi = reinterpret_cast<uint16_t*>(host.data() + u.off_ahi);
            uint16_t* lo = reinterpret_cast<uint16_t*>(host.data() + u.off_alo);
            for (int j = 0; j < u.a_chunks; ++j)
                for (int b = 0; b < 8; ++b)
                    for (int d = 0; d < 8; ++d) {
                        const long idx = (long)u.W + 127 - (8L * j + b + d);
                        const double h = (idx >= 0 && idx < u.L) ? std::ldexp(u.taps[idx], sh) : 0.0;
                        uint16_t vh, vl;
                        if (u.tc_mode == FIR_TC_FP16_SPLIT) {
                            vh = f2h((float)h);
                            vl = f2h((float)(h - h2d(vh)));
                        } else {
                            vh = f2bf((float)h);
                            vl = f2bf((float)(h - (double)bf2f(vh)));
                        }
                        hi[(j * 8 + b) * 8 + d] = vh;
                        lo[(j * 8 + b) * 8 + d] = vl;
                    }
        }
    }
    if (p->spectral) {
        fill_fft_tables(p->spec_fir, host.data());  // the chain's spectrum follows on the device
        const int M = p->spec_fir.fft_M;
        double2* zt = reinterpret_cast<double2*>(host.data() + p->off_spec_z);
        for (int k = 0; k < M; ++k) {
            const double ang = -2.0 * M_PI * (double)k / (double)M;
            zt[k] = make_double2(std::cos(ang), std::sin(ang));
        }
    }
    else if (p->use_chain)
        fill_fft_tables(p->chain, host.data());
    for (int32_t i = 0; i < nst; ++i) {
        float* d = reinterpret_cast<float*>(host.data() + p->plain[i].off);
        if (st[i].kind == TFX_STAGE_SOS) {
            for (int r = 0; r < st[i].n; ++r) {
                double row[5];
                normalise_row(st[i].coef + 6 * r, row);
                sec_device_coefs(row, d + 8 * r);
            }
        } else {
            for (int k = 0; k < st[i].n; ++k) d[k] = (float)st[i].coef[k];
        }
    }

    if (upload) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return TFX_ERR_CUDA;
        if (cudaMalloc(&p->dconst, host.size()) != cudaSuccess) return TFX_ERR_NOMEM;
        if (cudaMemcpy(p->dconst, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return TFX_ERR_CUDA;
        if (cudaMalloc(&p->dstatus, sizeof(int)) != cudaSuccess) return TFX_ERR_NOMEM;
        if (cudaMemset(p->dstatus, 0, sizeof(int)) != cudaSuccess) return TFX_ERR_CUDA;
        for (HostUnit& u : p->units) {
            if (u.fft) {
                if (prepare_fir_fft(u.fft_M) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
                continue;
            }
            if (u.seg) {
                if (prepare_sos_tc() != cudaSuccess) return TFX_ERR_UNSUPPORTED;
                continue;
            }
            if (u.tc) {
                if (u.tc_variant == 1) {
                    if (prepare_fir_tc_ws(u.tc_smem_ws) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
                } else if (u.tc_variant == 2) {
                    if (prepare_fir_tc_long(u.tc_smem_ws) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
                } else if (prepare_fir_tc(u.tc_smem) != cudaSuccess) {
                    return TFX_ERR_UNSUPPORTED;
                }
                continue;
            }
            UnitConst k{};
            k.S = u.S;
            k.L = u.L;
            k.H = u.L > 0 ? u.L - 1 : 0;
            k.nkb = u.nkb;
            if (prepare_unit(k) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
            if (p->train && u.S > 0 && prepare_sos_bwd(u.S) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
        }
        if (p->train && !(p->flags & TFX_PLAN_FIR_CUDA_CORES)) {
            for (HostUnit& u : p->units)
                if (u.L > 0 && prepare_fir_dh_tc() != cudaSuccess) return TFX_ERR_UNSUPPORTED;
        }
        if (p->use_chain && prepare_fir_fft(p->chain.fft_M) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
        if (p->spectral) {
            if (prepare_spectral(p->chain.fft_m) != cudaSuccess) return TFX_ERR_UNSUPPORTED;
            if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess)
                return TFX_ERR_CUDA;
            if (launch_chain_spectrum(reinterpret_cast<const double*>(p->dconst + p->off_spec_raw), p->chain_S,
                                      reinterpret_cast<const float2*>(p->dconst + p->spec_fir.off_H),
                                      reinterpret_cast<const double2*>(p->dconst + p->off_spec_z),
                                      p->chain.fft_m, reinterpret_cast<float2*>(p->dconst + p->chain.off_H),
                                      nullptr) != cudaSuccess ||
                cudaStreamSynchronize(nullptr) != cudaSuccess)
                return TFX_ERR_CUDA;
        }
    }

    // workspace layout
    const int64_t ntt = p->N > 0 ? (p->N + TILE - 1) / TILE : 0;
    size_t hdr = 0, tails = 0, zbytes = 0;
    for (HostUnit& u : p->units) {
        u.ntt = ntt;
        if (u.tc) {
            u.ntt = p->N > 0 ? (p->N + 128 * u.NB - 1) / (128 * u.NB) : 0;
            continue;
        }
        if (u.fft) {
            u.ntt = p->N > 0 ? (p->N + u.fft_B - 1) / u.fft_B : 0;
            if (u.fft_P > 0)  // segment spectra of every channel pair, in the scratch region
                zbytes = std::max(zbytes, align_up((size_t)((p->C + 1) / 2) * (size_t)u.ntt * u.fft_M * sizeof(float2)));
            continue;
        }
        // (a tensor-core cascade unit keeps the look-back fields below too: a
        // coefficient update switches the unit to that scan)
        if (u.warp) u.ntt = p->N > 0 ? (p->N + WARP_TILE - 1) / WARP_TILE : 0;
        const int H = u.L > 0 ? u.L - 1 : 0;
        u.tail_len = u.L > 0 ? (H < TILE ? H : TILE) : 0;
        const int64_t tiles = p->C * u.ntt;
        if (tiles > (int64_t)INT32_MAX) return TFX_ERR_UNSUPPORTED;
        u.flags_bytes = align_up((size_t)tiles * sizeof(unsigned));
        u.vals_bytes = (size_t)tiles * u.S * sizeof(Carry);
        u.tails_bytes = (size_t)tiles * u.tail_len * sizeof(float);
        // header = ticket, tail flags and carries: all reset per execution
        hdr = std::max(hdr, align_up(ALIGN + u.flags_bytes + u.vals_bytes));
        tails = std::max(tails, align_up(u.tails_bytes));
    }
    p->scratch_hdr = hdr;
    p->scratch_bytes = std::max(hdr + tails, zbytes);
    p->buf_bytes = align_up((size_t)p->C * (size_t)p->N * sizeof(float));
    size_t nbuf = p->units.size() > 2 ? 2 : (p->units.size() == 2 ? 1 : 0);
    if (p->units.size() == 1) {
        // input copy for in-place operation: the unit reads other tiles' or segments' input
        const HostUnit& u0 = p->units[0];
        if (u0.tc || (u0.fft && u0.fft_P == 0) || (u0.seg && u0.seg_P > 1 && u0.seg_D > 0)) nbuf = 1;
    }
    if (p->use_chain) {
        p->chain.ntt = p->N > 0 ? (p->N + p->chain.fft_B - 1) / p->chain.fft_B : 0;
        nbuf = std::max<size_t>(nbuf, 1);  // input copy for in-place operation
    }
    p->ws_fused = p->scratch_bytes + nbuf * p->buf_bytes;
    p->ws_plain = (nst > 0 ? 2 : 0) * p->buf_bytes;

    if (p->train && p->spectral) {
        // nothing saved (the backward reads x); backward workspace: the
        // correlation CTAs' partial spectra, their FP64 sum, the FIR taps'
        // gradient spectrum, the section-gradient blocks' partial sums and a
        // copy of the gradient for an in-place input gradient
        const int M = p->chain.fft_M;
        const int64_t items = (p->C + 1) / 2 * p->chain.ntt;
        p->spec_grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)p->sm_count *
                                                                               xcorr_ctas_per_sm(p->chain.fft_m)));
        p->saved_bytes = 0;
        p->b_sp_part = 0;
        p->b_sp_P = align_up((size_t)p->spec_grid * M * sizeof(float2));
        p->b_sp_w = p->b_sp_P + align_up((size_t)M * sizeof(double2));
        p->b_sp_gs = p->b_sp_w + align_up((size_t)M * sizeof(float2));
        p->b_gbuf = p->b_sp_gs + align_up(chain_grads_scratch_bytes(p->chain.fft_m, p->chain_S));
        p->bws_bytes = p->b_gbuf + p->buf_bytes;
    } else if (p->train) {
        // saved for the backward: the input of every unit after the first (the
        // first unit's input is x itself) and each cascade's chunk-start states
        p->nch = p->N > 0 ? (p->N + T_CHUNK - 1) / T_CHUNK : 0;
        size_t so = 0;
        for (size_t i = 0; i < p->units.size(); ++i) {
            HostUnit& u = p->units[i];
            if (i > 0) {
                u.off_act = so;
                so = align_up(so + p->buf_bytes);
            }
            if (u.S > 0) {
                u.off_ckpt = so;
                so = align_up(so + (size_t)p->C * u.S * p->nch * sizeof(float2));
            }
        }
        p->saved_bytes = so;
        // backward workspace: the forward scratch (FIR units run their forward
        // kernels on the reversed gradient), the reverse look-back scratch,
        // per-tile / per-block FP32 partials, FP64 column sums, two gradient buffers
        size_t scan = 0, part = 0, tmp = 0;
        for (const HostUnit& u : p->units) {
            if (u.S > 0) {
                const size_t tiles = (size_t)p->C * (size_t)u.ntt;
                scan = std::max(scan, align_up(ALIGN + tiles * u.S * sizeof(Carry)));
                part = std::max(part, align_up(tiles * u.S * 5 * sizeof(float)));
                tmp = std::max(tmp, align_up((size_t)u.S * 5 * sizeof(double)));
            } else if (u.L > 0) {
                size_t rows = (size_t)fir_dh_rows(p->C, p->N);
                if (!(p->flags & TFX_PLAN_FIR_CUDA_CORES)) {
                    int G, nwin, LW, NQ;
                    fir_dh_tc_geometry(p->C, p->N, u.L, p->sm_count, &G, &nwin, &LW, &NQ);
                    rows = (size_t)G;
                }
                part = std::max(part, align_up(rows * u.L * sizeof(float)));
            }
        }
        p->b_scan = p->scratch_bytes;
        p->b_part = p->b_scan + scan;
        p->b_tmp = p->b_part + part;
        p->b_gbuf = p->b_tmp + tmp;
        p->bws_bytes = p->b_gbuf + 2 * p->buf_bytes;
    }
    return TFX_OK;
}

bool ranges_overlap_not_equal(const float* x, const float* y, int64_t C, int64_t N, int64_t ld) {
    if (x == y || C == 0 || N == 0) return false;
    const char* xb = reinterpret_cast<const char*>(x);
    const char* yb = reinterpret_cast<const char*>(y);
    const size_t span = ((size_t)(C - 1) * (size_t)ld + (size_t)N) * sizeof(float);
    return xb < yb + span && yb < xb + span;
}

// Launch unit i for channels [c0, c0 + Cg) reading `in` (row stride ldin) and
// writing `out` (row stride ldout).  copy_buf ([Cg x N] floats) takes a copy
// of the input when a unit that reads other tiles' or segments' input runs
// in place; callers without one (the training forward and backward) never
// run such a unit in place: their inputs and outputs are distinct buffers
// (x != y is required, intermediates go to the saved buffer or to the
// gradient buffers), and trainable plans route cascades to the warp-tile
// scan, never to segments (build_plan: u.warp for p->train), which an
// assert in choose_segments' caller restates.
int launch_unit_range(tfx_plan* p, const HostUnit& u, const float* in, int64_t ldin, float* out, int64_t ldout,
                      int64_t c0, int64_t Cg, char* scratch, float* copy_buf, cudaStream_t s, float2* ckpt = nullptr) {
    in += c0 * ldin;
    out += c0 * ldout;
    if (u.fft) {
        FirFftArgs f{};
        f.x = in;
        f.ldx = ldin;
        f.y = out;
        f.ldy = ldout;
        // single-block: blocks read their predecessors' input, so an in-place
        // call copies it first; partitioned: every segment is transformed
        // before any output is written
        if (f.x == f.y && u.fft_P == 0) {
            if (launch_copy_rows(f.x, copy_buf, Cg, p->N, f.ldx, p->N, s) != cudaSuccess) return TFX_ERR_CUDA;
            f.x = copy_buf;
            f.ldx = p->N;
        }
        f.C = Cg;
        f.N = p->N;
        f.L = u.L;
        f.M = u.fft_M;
        f.m = u.fft_m;
        f.B = u.fft_B;
        f.P = u.fft_P;
        f.nbpc = u.ntt;
        f.nb = (u.fft_P > 0 ? (Cg + 1) / 2 : Cg) * u.ntt;
        f.Z = reinterpret_cast<float2*>(scratch);
        f.H = reinterpret_cast<const float2*>(p->dconst + u.off_H);
        f.tw = reinterpret_cast<const float2*>(p->dconst + u.off_tw);
        return launch_fir_fft(f, s) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
    }
    if (u.tc) {
        FirTcArgs f{};
        f.x = in;
        f.ldx = ldin;
        f.y = out;
        f.ldy = ldout;
        if (f.x == f.y) {  // the halo is read from other tiles' input: copy it first
            if (launch_copy_rows(f.x, copy_buf, Cg, p->N, f.ldx, p->N, s) != cudaSuccess) return TFX_ERR_CUDA;
            f.x = copy_buf;
            f.ldx = p->N;
        }
        f.C = Cg;
        f.N = p->N;
        f.ntt = u.ntt;
        f.L = u.L;
        f.W = u.W;
        f.nK = u.nK;
        f.NB = u.NB;
        f.rows = u.rows;
        f.tmem_cols = u.tmem_cols;
        f.a_chunks = u.a_chunks;
        f.mode = u.tc_mode;
        f.tap_unscale = u.tap_unscale;
        f.persistent = u.tc_variant;
        f.grid = p->sm_count;
        f.a_hi = reinterpret_cast<const uint4*>(p->dconst + u.off_ahi);
        f.a_lo = reinterpret_cast<const uint4*>(p->dconst + u.off_alo);
        f.status = p->dstatus;
        return launch_fir_tc(f, s) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
    }
    if (u.seg) {
        SegArgs g{};
        g.x = in;
        g.ldx = ldin;
        g.y = out;
        g.ldy = ldout;
        g.C = Cg;
        g.N = p->N;
        g.S = u.S;
        g.gain = 1.0f;
        g.coef = reinterpret_cast<const float*>(p->dconst + u.off_coef);
        g.Lseg = u.seg_len;
        g.P = u.seg_P;
        g.D = u.seg_D;
        if (g.x == g.y && g.P > 1 && g.D > 0) {  // warm-ups read the preceding segment's input: copy it first
            if (!copy_buf) return TFX_ERR_INVALID;
            if (launch_copy_rows(g.x, copy_buf, Cg, p->N, g.ldx, p->N, s) != cudaSuccess) return TFX_ERR_CUDA;
            g.x = copy_buf;
            g.ldx = p->N;
        }
        const char* t = p->dconst + u.off_tc;
        g.a1 = reinterpret_cast<const uint4*>(t);
        g.a2 = reinterpret_cast<const uint4*>(t + u.tc_a1.size());
        g.rowinv = reinterpret_cast<const float*>(t + u.tc_a1.size() + u.tc_a2.size());
        g.phib = g.rowinv + u.tc_rowinv.size();
        g.status = p->dstatus;
        return launch_sos_tc(g, p->sm_count, s) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
    }
    UnitArgs a{};
    a.x = in;
    a.ldx = ldin;
    a.y = out;
    a.ldy = ldout;
    a.C = Cg;
    a.N = p->N;
    a.ntt = u.ntt;
    a.k.S = u.S;
    a.k.L = u.L;
    a.k.H = u.L > 0 ? u.L - 1 : 0;
    a.k.nkb = u.nkb;
    a.k.gain = 1.0f;
    a.k.coef = reinterpret_cast<const float*>(p->dconst + u.off_coef);
    a.k.pw = reinterpret_cast<const float4*>(p->dconst + u.off_pw);
    a.k.taps = reinterpret_cast<const float*>(p->dconst + u.off_taps);
    a.k.pw64 = u.hiq ? reinterpret_cast<const double4*>(p->dconst + u.off_pw64) : nullptr;
    a.sc.ticket = reinterpret_cast<unsigned*>(scratch);
    a.sc.flags = reinterpret_cast<unsigned*>(scratch + ALIGN);
    a.sc.carry = reinterpret_cast<Carry*>(scratch + ALIGN + u.flags_bytes);
    a.sc.tails = reinterpret_cast<float*>(scratch + p->scratch_hdr);
    a.sc.tail_len = u.tail_len;
    a.status = p->dstatus;
    a.drop_tile = (p->flags & TFX_PLAN_TEST_DROP_PUBLISH) ? 0 : -1;
    a.ckpt = u.warp ? ckpt : nullptr;
    a.nch = p->nch;
    if (cudaMemsetAsync(scratch, 0, ALIGN + u.flags_bytes + u.vals_bytes, s) != cudaSuccess) return TFX_ERR_CUDA;
    return (u.warp ? launch_sos_warp(a, s) : launch_unit(a, s)) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
}

int exec_fused(tfx_plan* p, const float* x, float* y, void* ws, cudaStream_t s) {
    char* w = static_cast<char*>(ws);
    const int nu = (int)p->units.size();
    if (nu == 0) {
        if (x != y) {
            if (launch_copy_rows(x, y, p->C, p->N, p->ld, p->ld, s) != cudaSuccess) return TFX_ERR_CUDA;
        }
        return TFX_OK;
    }
    char* scratch = w;
    float* buf[2] = {reinterpret_cast<float*>(w + p->scratch_bytes),
                     reinterpret_cast<float*>(w + p->scratch_bytes + p->buf_bytes)};
    if (p->use_chain) return launch_unit_range(p, p->chain, x, p->ld, y, p->ld, 0, p->C, scratch, buf[0], s);
    for (int i = 0; i < nu; ++i) {
        const float* in = i == 0 ? x : buf[(i - 1) & 1];
        const int64_t ldin = i == 0 ? p->ld : p->N;
        float* out = i == nu - 1 ? y : buf[i & 1];
        const int64_t ldout = i == nu - 1 ? p->ld : p->N;
        const int rc = launch_unit_range(p, p->units[i], in, ldin, out, ldout, 0, p->C, scratch, buf[0], s);
        if (rc != TFX_OK) return rc;
    }
    return TFX_OK;
}

int exec_plain(tfx_plan* p, const float* x, float* y, void* ws, cudaStream_t s) {
    const int ns = (int)p->plain.size();
    for (const PlainStage& st : p->plain)
        if (st.kind == TFX_STAGE_SOS && st.n > 64) return TFX_ERR_UNSUPPORTED;
    if (ns == 0) {
        if (x != y && launch_copy_rows(x, y, p->C, p->N, p->ld, p->ld, s) != cudaSuccess) return TFX_ERR_CUDA;
        return TFX_OK;
    }
    float* buf[2] = {reinterpret_cast<float*>(ws), reinterpret_cast<float*>(static_cast<char*>(ws) + p->buf_bytes)};
    const float* cur = x;
    int64_t ldc = p->ld;
    for (int i = 0; i < ns; ++i) {
        const PlainStage& st = p->plain[i];
        // the last stage writes y directly unless that would be an in-place FIR
        const bool direct = i == ns - 1 && !(st.kind == TFX_STAGE_FIR && cur == y);
        float* out = direct ? y : buf[i & 1];
        int64_t ldo = direct ? p->ld : p->N;
        if (st.kind == TFX_STAGE_SOS) {
            if (launch_plain_sos(cur, out, p->C, p->N, ldc, ldo, st.n,
                                 reinterpret_cast<const float*>(p->dconst + st.off), s) != cudaSuccess)
                return TFX_ERR_CUDA;
        } else {
            if (launch_plain_fir(cur, out, p->C, p->N, ldc, ldo, st.n,
                                 reinterpret_cast<const float*>(p->dconst + st.off), s) != cudaSuccess)
                return TFX_ERR_CUDA;
        }
        cur = out;
        ldc = ldo;
    }
    if (cur != y && launch_copy_rows(cur, y, p->C, p->N, ldc, p->ld, s) != cudaSuccess) return TFX_ERR_CUDA;
    return TFX_OK;
}

// Training forward: the fused units of a trainable plan, with every
// intermediate written to the saved buffer (the backward reads it) and every
// cascade storing its chunk-start states there.
int exec_train(tfx_plan* p, const float* x, float* y, char* saved, void* ws, cudaStream_t s) {
    char* scratch = static_cast<char*>(ws);
    if (p->spectral) return launch_unit_range(p, p->chain, x, p->ld, y, p->ld, 0, p->C, scratch, nullptr, s);
    const int nu = (int)p->units.size();
    if (nu == 0) return launch_copy_rows(x, y, p->C, p->N, p->ld, p->ld, s) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
    for (int i = 0; i < nu; ++i) {
        const HostUnit& u = p->units[i];
        const float* in = i == 0 ? x : reinterpret_cast<const float*>(saved + u.off_act);
        const int64_t ldin = i == 0 ? p->ld : p->N;
        float* out = i == nu - 1 ? y : reinterpret_cast<float*>(saved + p->units[i + 1].off_act);
        const int64_t ldout = i == nu - 1 ? p->ld : p->N;
        float2* ck = u.S > 0 ? reinterpret_cast<float2*>(saved + u.off_ckpt) : nullptr;
        const int rc = launch_unit_range(p, p->units[i], in, ldin, out, ldout, 0, p->C, scratch, nullptr, s, ck);
        if (rc != TFX_OK) return rc;
    }
    return TFX_OK;
}

// The spectral input gradient: the chain over g in reverse time by the
// forward's FFT kernel (after a copy of g when dx is g: blocks read their
// neighbours' gradient samples), on stream s.
int spectral_dx(tfx_plan* p, const float* g, float* dx, char* ws, cudaStream_t s, bool count_only, int* nlaunch) {
    const HostUnit& c = p->chain;
    const float* gin = g;
    int64_t ldg = p->ld;
    if (dx == g) {  // blocks read their neighbours' gradient samples
        float* gb = reinterpret_cast<float*>(ws + p->b_gbuf);
        ++*nlaunch;
        if (!count_only && launch_copy_rows(g, gb, p->C, p->N, p->ld, p->N, s) != cudaSuccess) return TFX_ERR_CUDA;
        gin = gb;
        ldg = p->N;
    }
    FirFftArgs f{};
    f.x = gin;
    f.ldx = ldg;
    f.y = dx;
    f.ldy = p->ld;
    f.C = p->C;
    f.N = p->N;
    f.L = c.L;
    f.M = c.fft_M;
    f.m = c.fft_m;
    f.B = c.fft_B;
    f.P = 0;
    f.nbpc = c.ntt;
    f.nb = p->C * c.ntt;
    f.H = reinterpret_cast<const float2*>(p->dconst + c.off_H);
    f.tw = reinterpret_cast<const float2*>(p->dconst + c.off_tw);
    f.rev = 1;
    ++*nlaunch;
    if (!count_only && launch_fir_fft(f, s) != cudaSuccess) return TFX_ERR_CUDA;
    return TFX_OK;
}

// Backward of a spectral plan.  Coefficient gradients: the correlation
// CTAs accumulate the block cross-spectra of g and x, their sum P (FP64)
// gives the section gradients by the closed-form derivative spectra and the
// FIR taps' gradient by one inverse transform, and the section sums map to
// the raw rows (the a0 chain rule) in one launch.  Input gradient: the chain
// applied to g in reverse time (its transpose), by the forward's kernel with
// reversed rows, after the correlation (which reads g) when dx is g.
// The backward of a spectral plan after the correlation partials are in
// the workspace (ws + b_sp_part, p->spec_grid rows): dL/dx on the side
// stream (it only needs g), the partials' sum P, the derivative spectra's
// section and FIR-tap gradients, the a0 chain rule; the caller's stream
// waits for dL/dx at the end.
int spectral_grads_from_partials(tfx_plan* p, const float* g, float* dx, double* dcoef, char* ws, cudaStream_t s,
                                 bool count_only, int* nlaunch) {
    int nl = 0;
#define TFX_LAUNCH(call)                                               \
    do {                                                               \
        ++nl;                                                          \
        if (!count_only && (call) != cudaSuccess) return TFX_ERR_CUDA; \
    } while (0)
    const HostUnit& c = p->chain;
    const int m = c.fft_m, M = c.fft_M;
    const float2* tw = reinterpret_cast<const float2*>(p->dconst + c.off_tw);
    double2* P = reinterpret_cast<double2*>(ws + p->b_sp_P);
    float2* part = reinterpret_cast<float2*>(ws + p->b_sp_part);
    if (dx) {
        // dx only needs g (complete by now): it runs on the side stream
        // beside the small gradient kernels below
        if (!count_only && (cudaEventRecord(p->ev_fork, s) != cudaSuccess ||
                            cudaStreamWaitEvent(p->side, p->ev_fork, 0) != cudaSuccess))
            return TFX_ERR_CUDA;
        const int rc = spectral_dx(p, g, dx, ws, p->side, count_only, &nl);
        if (rc != TFX_OK) return rc;
        if (!count_only && cudaEventRecord(p->ev_join, p->side) != cudaSuccess) return TFX_ERR_CUDA;
    }
    TFX_LAUNCH(launch_xcorr_reduce(part, p->spec_grid, M, P, s));
    const double* raw = reinterpret_cast<const double*>(p->dconst + p->off_spec_raw);
    nl += p->spec_nfir ? 2 : 1;
    if (!count_only &&
        launch_chain_grads(m, P, raw, p->chain_S, reinterpret_cast<const float2*>(p->dconst + p->spec_fir.off_H),
                           reinterpret_cast<const double2*>(p->dconst + p->off_spec_z), tw, p->spec_fir.L,
                           ws + p->b_sp_gs, reinterpret_cast<float2*>(ws + p->b_sp_w),
                           p->spec_nfir ? dcoef + p->spec_fir_dst : nullptr, s) != cudaSuccess)
        return TFX_ERR_CUDA;
    TFX_LAUNCH(launch_spectral_finalize(m, ws + p->b_sp_gs, p->chain_S, raw,
                                        reinterpret_cast<const int64_t*>(p->dconst + p->off_spec_dst), dcoef, s));
    // join: the caller's stream continues once the input gradient is done
    if (dx && !count_only && cudaStreamWaitEvent(s, p->ev_join, 0) != cudaSuccess) return TFX_ERR_CUDA;
#undef TFX_LAUNCH
    if (nlaunch) *nlaunch += nl;
    return TFX_OK;
}

int run_backward_spectral(tfx_plan* p, const float* x, const float* g, float* dx, double* dcoef, char* ws,
                          cudaStream_t s, bool count_only, int* nlaunch) {
    int nl = 0;
    const HostUnit& c = p->chain;
    if (dcoef) {
        XcorrArgs a{};
        a.x = x;
        a.g = g;
        a.ldx = p->ld;
        a.ldg = p->ld;
        a.C = p->C;
        a.N = p->N;
        a.J = c.L - 1;
        a.B = c.fft_B;
        a.nbpc = c.ntt;
        a.items = (p->C + 1) / 2 * c.ntt;
        a.tw = reinterpret_cast<const float2*>(p->dconst + c.off_tw);
        a.part = reinterpret_cast<float2*>(ws + p->b_sp_part);
        ++nl;
        if (!count_only && launch_chain_xcorr(c.fft_m, a, p->spec_grid, s) != cudaSuccess) return TFX_ERR_CUDA;
        const int rc = spectral_grads_from_partials(p, g, dx, dcoef, ws, s, count_only, &nl);
        if (rc != TFX_OK) return rc;
    }
    if (dx && !dcoef) {
        const int rc = spectral_dx(p, g, dx, ws, s, count_only, &nl);
        if (rc != TFX_OK) return rc;
    }
    if (nlaunch) *nlaunch = nl;
    return TFX_OK;
}

// Backward over the units, last to first.  Between units the gradient is
// kept either in time order or time-reversed: an FIR's input gradient is the
// same FIR applied to the reversed gradient (FIR^T = J FIR J, J the time
// reversal), so FIR units take and produce the reversed form, and a cascade
// in front of an FIR writes it reversed.  With count_only nothing is enqueued
// and *nlaunch receives the number of kernels a real call launches.
int run_backward(tfx_plan* p, const float* x, const float* g, float* dx, double* dcoef, const char* saved, char* ws,
                 cudaStream_t s, bool count_only, int* nlaunch) {
    if (p->spectral) return run_backward_spectral(p, x, g, dx, dcoef, ws, s, count_only, nlaunch);
    int nl = 0;
#define TFX_LAUNCH(call)                                                     \
    do {                                                                     \
        ++nl;                                                                \
        if (!count_only && (call) != cudaSuccess) return TFX_ERR_CUDA;       \
    } while (0)
    const int nu = (int)p->units.size();
    const int64_t C = p->C, N = p->N;
    float* gbuf[2] = {reinterpret_cast<float*>(ws + p->b_gbuf), reinterpret_cast<float*>(ws + p->b_gbuf + p->buf_bytes)};
    float* part = reinterpret_cast<float*>(ws + p->b_part);
    double* tmp = reinterpret_cast<double*>(ws + p->b_tmp);
    const float* gcur = g;
    int64_t ldg = p->ld;
    bool grev = false;
    int cur = -1;  // gradient buffer holding gcur (-1: the caller's g)
    if (nu == 0 && dx && dx != g) TFX_LAUNCH(launch_copy_rows(g, dx, C, N, p->ld, p->ld, s));
    for (int i = nu - 1; i >= 0; --i) {
        const HostUnit& u = p->units[i];
        const float* uin = i == 0 ? x : reinterpret_cast<const float*>(saved + u.off_act);
        const int64_t ldu = i == 0 ? p->ld : N;
        int nxt = cur == 0 ? 1 : 0;
        if (u.S > 0) {
            BwdArgs a{};
            a.u0 = uin;
            a.ldu = ldu;
            a.g = gcur;
            a.ldg = ldg;
            a.g_rev = grev ? 1 : 0;
            if (i == 0) {
                a.gout = dx;
                a.ldo = p->ld;
                a.out_rev = 0;
            } else {
                a.gout = gbuf[nxt];
                a.ldo = N;
                a.out_rev = p->units[i - 1].S == 0 ? 1 : 0;
            }
            a.ckpt = reinterpret_cast<const float2*>(saved + u.off_ckpt);
            a.nch = p->nch;
            a.C = C;
            a.N = N;
            a.ntt = u.ntt;
            a.k.S = u.S;
            a.k.gain = 1.0f;
            a.k.coef = reinterpret_cast<const float*>(p->dconst + u.off_coef);
            a.k.pw = reinterpret_cast<const float4*>(p->dconst + u.off_pw);
            a.ticket = reinterpret_cast<unsigned*>(ws + p->b_scan);
            a.carry = reinterpret_cast<Carry*>(ws + p->b_scan + ALIGN);
            a.part = part;
            a.status = p->dstatus;
            const int64_t tiles = C * u.ntt;
            if (!count_only &&
                cudaMemsetAsync(ws + p->b_scan, 0, ALIGN + (size_t)tiles * u.S * sizeof(Carry), s) != cudaSuccess)
                return TFX_ERR_CUDA;
            TFX_LAUNCH(launch_sos_bwd(a, s));
            if (dcoef) {
                TFX_LAUNCH(launch_colsum(part, tiles, u.S * 5, tmp, s));
                TFX_LAUNCH(launch_sos_grad_finalize(tmp, u.S, reinterpret_cast<const double*>(p->dconst + u.off_raw),
                                                    reinterpret_cast<const int64_t*>(p->dconst + u.off_dst), dcoef,
                                                    s));
            }
            if (i > 0) {
                gcur = gbuf[nxt];
                ldg = N;
                grev = a.out_rev != 0;
                cur = nxt;
            }
        } else {
            const bool want_out = i > 0 || dx != nullptr;
            if (dcoef) {
                if (p->flags & TFX_PLAN_FIR_CUDA_CORES) {
                    TFX_LAUNCH(launch_fir_dh(gcur, ldg, grev ? 1 : 0, uin, ldu, C, N, u.L, u.Lp, part, s));
                    TFX_LAUNCH(launch_colsum(part, fir_dh_rows(C, N), u.L, dcoef + u.fir_dst, s));
                } else {
                    // the tap-gradient GEMM also writes the reversed gradient the
                    // input-gradient pass needs, so no separate flip follows
                    float* gf = (!grev && want_out) ? gbuf[nxt] : nullptr;
                    int G, nwin, LW, NQ;
                    fir_dh_tc_geometry(C, N, u.L, p->sm_count, &G, &nwin, &LW, &NQ);
                    TFX_LAUNCH(launch_fir_dh_tc(gcur, ldg, grev ? 1 : 0, uin, ldu, gf, C, N, u.L, p->sm_count, part,
                                                p->dstatus, s));
                    TFX_LAUNCH(launch_colsum(part, G, u.L, dcoef + u.fir_dst, s));
                    if (gf) {
                        gcur = gbuf[nxt];
                        ldg = N;
                        grev = true;
                        cur = nxt;
                    }
                }
            }
            if (!want_out) continue;
            nxt = cur == 0 ? 1 : 0;
            if (!grev) {
                TFX_LAUNCH(launch_flip_rows(gcur, gbuf[nxt], C, N, ldg, N, s));
                gcur = gbuf[nxt];
                ldg = N;
                grev = true;
                cur = nxt;
            }
            const int o = cur == 0 ? 1 : 0;
            ++nl;
            if (!count_only) {
                const int rc = launch_unit_range(p, p->units[i], gcur, N, gbuf[o], N, 0, C, ws, nullptr, s);
                if (rc != TFX_OK) return rc;
            }
            if (i == 0) {
                TFX_LAUNCH(launch_flip_rows(gbuf[o], dx, C, N, N, p->ld, s));
            } else {
                gcur = gbuf[o];
                ldg = N;
                cur = o;
            }
        }
    }
#undef TFX_LAUNCH
    if (nlaunch) *nlaunch = nl;
    return TFX_OK;
}

// Byte span of a [C x N] signal with row stride ld.
size_t signal_span(int64_t C, int64_t N, int64_t ld) {
    return C == 0 || N == 0 ? 0 : ((size_t)(C - 1) * (size_t)ld + (size_t)N) * sizeof(float);
}

bool bytes_overlap(const void* a, size_t na, const void* b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    const char* ab = static_cast<const char*>(a);
    const char* bb = static_cast<const char*>(b);
    return ab < bb + nb && bb < ab + na;
}

int check_exec_args(tfx_plan* p, const float* x, float* y, void* ws, size_t ws_bytes, size_t need) {
    if (!p) return TFX_ERR_INVALID;
    if (p->C > 0 && p->N > 0 && (!x || !y)) return TFX_ERR_INVALID;
    if (ranges_overlap_not_equal(x, y, p->C, p->N, p->ld)) return TFX_ERR_INVALID;
    if (need > 0) {
        if (!ws || ws_bytes < need) return TFX_ERR_WORKSPACE;
        if (reinterpret_cast<uintptr_t>(ws) % ALIGN != 0) return TFX_ERR_WORKSPACE;
    }
    return TFX_OK;
}

// ---------------------------------------------------------------------------
// one-shot plan cache

struct CacheEntry {
    tfx_plan* plan = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
};

std::mutex g_mu;
std::list<std::string> g_lru;
std::unordered_map<std::string, std::pair<CacheEntry, std::list<std::string>::iterator>> g_cache;
constexpr size_t CACHE_MAX = 32;

std::string cache_key(int64_t C, int64_t N, int64_t ld, const tfx_stage* st, int32_t nst, cudaStream_t s) {
    std::string k;
    auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
    put(&C, 8);
    put(&N, 8);
    put(&ld, 8);
    put(&s, sizeof(s));
    put(&nst, 4);
    for (int32_t i = 0; i < nst; ++i) {
        put(&st[i].kind, 4);
        put(&st[i].n, 4);
        const size_t cnt = st[i].kind == TFX_STAGE_SOS ? (size_t)st[i].n * 6 : (size_t)st[i].n;
        if (cnt) put(st[i].coef, cnt * sizeof(double));
    }
    return k;
}

void free_entry(CacheEntry& e) {
    if (e.ws) cudaFree(e.ws);
    tfx_plan_destroy(e.plan);
    e = CacheEntry();
}

int cached_plan(int64_t C, int64_t N, int64_t ld, const tfx_stage* st, int32_t nst, cudaStream_t s,
                CacheEntry* out) {
    const std::string key = cache_key(C, N, ld, st, nst, s);
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        g_lru.splice(g_lru.begin(), g_lru, it->second.second);
        *out = it->second.first;
        return TFX_OK;
    }
    CacheEntry e;
    int rc = tfx_plan_create(&e.plan, C, N, ld, st, nst, TFX_PLAN_DEFAULT);
    if (rc != TFX_OK) return rc;
    e.ws_bytes = tfx_plan_workspace_size(e.plan);
    if (e.ws_bytes > 0 && cudaMalloc(&e.ws, e.ws_bytes) != cudaSuccess) {
        free_entry(e);
        return TFX_ERR_NOMEM;
    }
    if (g_cache.size() >= CACHE_MAX) {
        const std::string& old = g_lru.back();
        auto oit = g_cache.find(old);
        free_entry(oit->second.first);
        g_cache.erase(oit);
        g_lru.pop_back();
    }
    g_lru.push_front(key);
    g_cache.emplace(key, std::make_pair(e, g_lru.begin()));
    *out = e;
    return TFX_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

int tfx_plan_create(tfx_plan** out, int64_t C, int64_t N, int64_t ld, const tfx_stage* st, int32_t nst,
                    uint32_t flags) {
    return plan_create_ex(out, C, N, ld, st, nst, flags, TC_MIN_TAPS);
}

}  // extern "C"

int tfx::plan_create_ex(tfx_plan** out, int64_t C, int64_t N, int64_t ld, const tfx_stage* st, int32_t nst,
                        uint32_t flags, int tc_min_taps, bool allow_hiq, const int32_t* compose_m) {
    if (!out) return TFX_ERR_INVALID;
    *out = nullptr;
    int rc = check_dims(C, N, ld);
    if (rc != TFX_OK) return rc;
    rc = validate_stages(st, nst);
    if (rc != TFX_OK) return rc;
    if (flags & ~(TFX_PLAN_FIR_CUDA_CORES | TFX_PLAN_UNFUSED | TFX_PLAN_FIR_BF16_PLAIN | TFX_PLAN_FIR_BF16_SPLIT |
                  TFX_PLAN_SCAN_WARP_TILES | TFX_PLAN_TRAINABLE | TFX_PLAN_FIR_FFT | TFX_PLAN_FIR_TC |
                  TFX_PLAN_FIR_FFT_LOG_MASK | TFX_PLAN_SCAN_LOOKBACK | TFX_PLAN_TEST_DROP_PUBLISH |
                  TFX_PLAN_NO_COMPOSE))
        return TFX_ERR_INVALID;
    tfx_plan* p = new (std::nothrow) tfx_plan();
    if (!p) return TFX_ERR_NOMEM;
    p->C = C;
    p->N = N;
    p->ld = ld;
    p->flags = flags;
    p->tc_min_taps = tc_min_taps > 0 ? tc_min_taps : TC_MIN_TAPS;
    p->allow_hiq = allow_hiq;
    if (compose_m) std::copy(compose_m, compose_m + 16, p->compose_m);
    rc = build_plan(p, st, nst, true);
    if (rc != TFX_OK) {
        tfx_plan_destroy(p);
        return rc;
    }
    *out = p;
    return TFX_OK;
}

extern "C" {

size_t tfx_plan_workspace_size(const tfx_plan* p) {
    if (!p) return 0;
    return p->ws_fused > p->ws_plain ? p->ws_fused : p->ws_plain;
}

int tfx_plan_launch_count(const tfx_plan* p) {
    if (!p) return -1;
    if (p->C == 0 || p->N == 0) return 0;
    if (p->use_chain) return 1;
    int n = 0;
    for (const HostUnit& u : p->units) n += u.fft && u.fft_P > 0 ? 2 : 1;
    return p->units.empty() ? 1 : n;
}

int tfx_plan_describe(const tfx_plan* p, char* buf, size_t len) {
    if (!p) return -1;
    std::string d;
    char item[160];
    if (p->spectral) {
        const HostUnit& c = p->chain;
        snprintf(item, sizeof item, "chain_spectral:S=%d,L=%d,D=%d,J=%d,M=%d,B=%d", p->chain_S, p->chain_L,
                 p->chain_D, c.L - 1, c.fft_M, c.fft_B);
        d = item;
    } else if (p->use_chain) {
        const HostUnit& c = p->chain;
        snprintf(item, sizeof item, "chain_fft:S=%d,L=%d,D=%d,Lc=%d,M=%d,B=%d", p->chain_S, p->chain_L, p->chain_D,
                 c.L, c.fft_M, c.fft_B);
        d = item;
    }
    for (const HostUnit& u : (p->use_chain ? std::vector<HostUnit>() : p->units)) {
        if (!d.empty()) d += ';';
        if (u.fft) {
            snprintf(item, sizeof item, "fir_fft:L=%d,M=%d,B=%d,P=%d", u.L, u.fft_M, u.fft_B, u.fft_P);
        } else if (u.tc) {
            snprintf(item, sizeof item, "fir_tc:L=%d,kernel=%s", u.L,
                     u.tc_variant == 1 ? "k_fir_tc_ws" : u.tc_variant == 2 ? "k_fir_tc_long" : "k_fir_tc");
        } else if (u.S > 0 && u.L > 0) {
            snprintf(item, sizeof item, "fused:S=%d,L=%d", u.S, u.L);
        } else if (u.S > 0 && u.seg) {
            snprintf(item, sizeof item, "cascade:S=%d,scan=tc,carry=fp32,segments=%lld,D=%d", u.S,
                     (long long)u.seg_P, u.seg_D);
        } else if (u.S > 0) {
            snprintf(item, sizeof item, "cascade:S=%d,scan=%s,carry=%s", u.S, u.warp ? "warp" : "block",
                     u.hiq ? "fp64" : "fp32");
        } else {
            snprintf(item, sizeof item, "fir:L=%d", u.L);
        }
        d += item;
    }
    if (buf && len > 0) {
        const size_t n = std::min(len - 1, d.size());
        memcpy(buf, d.data(), n);
        buf[n] = '\0';
    }
    return (int)d.size();
}

int tfx_plan_execute(tfx_plan* p, const float* x, float* y, void* ws, size_t ws_bytes, tfx_stream s) {
    const size_t need = p ? p->ws_fused : 0;
    int rc = check_exec_args(p, x, y, ws, ws_bytes, need);
    if (rc != TFX_OK) return rc;
    if (p->C == 0 || p->N == 0) return TFX_OK;
    return exec_fused(p, x, y, ws, reinterpret_cast<cudaStream_t>(s));
}

int tfx_plan_execute_plain(tfx_plan* p, const float* x, float* y, void* ws, size_t ws_bytes, tfx_stream s) {
    const size_t need = p ? p->ws_plain : 0;
    int rc = check_exec_args(p, x, y, ws, ws_bytes, need);
    if (rc != TFX_OK) return rc;
    if (p->C == 0 || p->N == 0) return TFX_OK;
    return exec_plain(p, x, y, ws, reinterpret_cast<cudaStream_t>(s));
}

int tfx_plan_get_error(tfx_plan* p) {
    if (!p || !p->dstatus) return TFX_ERR_INVALID;
    if (cudaDeviceSynchronize() != cudaSuccess) return TFX_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, p->dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TFX_ERR_CUDA;
    if (v != 0 && cudaMemset(p->dstatus, 0, sizeof(int)) != cudaSuccess) return TFX_ERR_CUDA;
    return v;
}

void tfx_plan_destroy(tfx_plan* p) {
    if (!p) return;
    if (p->dconst || p->dstatus) cudaDeviceSynchronize();
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->dconst) cudaFree(p->dconst);
    if (p->dstatus) cudaFree(p->dstatus);
    if (p->dsec) cudaFree(p->dsec);
    delete p;
}

size_t tfx_plan_saved_size(const tfx_plan* p) { return p && p->train ? p->saved_bytes : 0; }

size_t tfx_plan_backward_workspace_size(const tfx_plan* p) { return p && p->train ? p->bws_bytes : 0; }

int64_t tfx_plan_coef_count(const tfx_plan* p) { return p ? p->ncoef : -1; }

int tfx_plan_forward_train(tfx_plan* p, const float* x, float* y, void* saved, size_t saved_bytes, void* ws,
                           size_t ws_bytes, tfx_stream s) {
    if (!p || !p->train) return TFX_ERR_INVALID;
    int rc = check_exec_args(p, x, y, ws, ws_bytes, p->ws_fused);
    if (rc != TFX_OK) return rc;
    if (p->C == 0 || p->N == 0) return TFX_OK;
    if (x == y) return TFX_ERR_INVALID;  // the backward reads x again
    if (p->saved_bytes > 0 &&
        (!saved || saved_bytes < p->saved_bytes || reinterpret_cast<uintptr_t>(saved) % ALIGN != 0))
        return TFX_ERR_WORKSPACE;
    const size_t span = signal_span(p->C, p->N, p->ld);
    if (bytes_overlap(saved, p->saved_bytes, x, span) || bytes_overlap(saved, p->saved_bytes, y, span))
        return TFX_ERR_INVALID;
    return exec_train(p, x, y, static_cast<char*>(saved), ws, reinterpret_cast<cudaStream_t>(s));
}

int tfx_plan_forward_train_mse(tfx_plan* p, const float* x, float* y, const float* target, float* g, double* loss,
                               void* saved, size_t saved_bytes, void* ws, size_t ws_bytes, tfx_stream s) {
    if (!p || !p->train || !loss) return TFX_ERR_INVALID;
    int rc = check_exec_args(p, x, y, ws, ws_bytes, p->ws_fused);
    if (rc != TFX_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    if (p->C == 0 || p->N == 0)
        return cudaMemsetAsync(loss, 0, sizeof(double), st) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
    if (x == y || !target || !g) return TFX_ERR_INVALID;
    const size_t span = signal_span(p->C, p->N, p->ld);
    // g may take the target's place; nothing else may overlap
    if (bytes_overlap(g, span, x, span) || bytes_overlap(g, span, y, span) ||
        (g != target && bytes_overlap(g, span, target, span)) || bytes_overlap(target, span, y, span) ||
        bytes_overlap(loss, sizeof(double), g, span) || bytes_overlap(loss, sizeof(double), y, span))
        return TFX_ERR_INVALID;
    if (p->saved_bytes > 0 &&
        (!saved || saved_bytes < p->saved_bytes || reinterpret_cast<uintptr_t>(saved) % ALIGN != 0))
        return TFX_ERR_WORKSPACE;
    if (bytes_overlap(saved, p->saved_bytes, x, span) || bytes_overlap(saved, p->saved_bytes, y, span))
        return TFX_ERR_INVALID;
    const double inv = 1.0 / ((double)p->C * (double)p->N);
    if (!p->spectral) {  // the units, then the loss kernel
        rc = exec_train(p, x, y, static_cast<char*>(saved), ws, st);
        if (rc != TFX_OK) return rc;
        return launch_mse(y, target, g, p->C, p->N, p->ld, loss, st) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
    }
    // spectral route: one FFT launch writes y, g and the loss
    if (cudaMemsetAsync(loss, 0, sizeof(double), st) != cudaSuccess) return TFX_ERR_CUDA;
    const HostUnit& c = p->chain;
    FirFftArgs f{};
    f.x = x;
    f.ldx = p->ld;
    f.y = y;
    f.ldy = p->ld;
    f.C = p->C;
    f.N = p->N;
    f.L = c.L;
    f.M = c.fft_M;
    f.m = c.fft_m;
    f.B = c.fft_B;
    f.P = 0;
    f.nbpc = c.ntt;
    f.nb = p->C * c.ntt;
    f.H = reinterpret_cast<const float2*>(p->dconst + c.off_H);
    f.tw = reinterpret_cast<const float2*>(p->dconst + c.off_tw);
    f.tgt = target;
    f.gout = g;
    f.loss = loss;
    f.gscale = (float)(2.0 * inv);
    f.lscale = inv;
    return launch_fir_fft(f, st) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
}

int tfx_plan_forward_train_mse_launch_count(const tfx_plan* p) {
    if (!p || !p->train) return -1;
    if (p->C == 0 || p->N == 0) return 0;
    return p->spectral ? 1 : tfx_plan_launch_count(p) + 1;
}

int tfx_plan_backward(tfx_plan* p, const float* x, const float* g, float* dx, double* dcoef, const void* saved,
                      size_t saved_bytes, void* ws, size_t ws_bytes, tfx_stream s) {
    if (!p || !p->train) return TFX_ERR_INVALID;
    if (!dx && !dcoef) return TFX_ERR_INVALID;
    const int64_t C = p->C, N = p->N;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    if (C == 0 || N == 0) {
        if (dcoef && p->ncoef > 0 && cudaMemsetAsync(dcoef, 0, (size_t)p->ncoef * sizeof(double), st) != cudaSuccess)
            return TFX_ERR_CUDA;
        return TFX_OK;
    }
    if (!x || !g) return TFX_ERR_INVALID;
    const size_t span = signal_span(C, N, p->ld);
    if (dx && (ranges_overlap_not_equal(g, dx, C, N, p->ld) || bytes_overlap(x, span, dx, span)))
        return TFX_ERR_INVALID;
    if (p->bws_bytes > 0 && (!ws || ws_bytes < p->bws_bytes || reinterpret_cast<uintptr_t>(ws) % ALIGN != 0))
        return TFX_ERR_WORKSPACE;
    if (p->saved_bytes > 0 &&
        (!saved || saved_bytes < p->saved_bytes || reinterpret_cast<uintptr_t>(saved) % ALIGN != 0))
        return TFX_ERR_WORKSPACE;
    return run_backward(p, x, g, dx, dcoef, static_cast<const char*>(saved), static_cast<char*>(ws), st, false,
                        nullptr);
}

int tfx_plan_backward_launch_count(const tfx_plan* p, int with_dx, int with_dcoef) {
    if (!p || !p->train) return -1;
    if (p->C == 0 || p->N == 0) return 0;
    int n = 0;
    // count_only: no pointer is dereferenced and nothing is enqueued
    float dummy_dx;
    double dummy_dc;
    run_backward(const_cast<tfx_plan*>(p), nullptr, nullptr, with_dx ? &dummy_dx : nullptr,
                 with_dcoef ? &dummy_dc : nullptr, nullptr, nullptr, nullptr, true, &n);
    return n;
}

int tfx_plan_train_step_mse(tfx_plan* p, const float* x, float* y, const float* target, float* g, double* loss,
                            float* dx, double* dcoef, void* saved, size_t saved_bytes, void* ws, size_t ws_bytes,
                            tfx_stream s) {
    if (!p || !p->train || !loss) return TFX_ERR_INVALID;
    const bool fused = p->spectral && dcoef && p->C > 0 && p->N > 0;
    if (!fused) {  // the two calls in order (each validates its own arguments)
        const int rc = tfx_plan_forward_train_mse(p, x, y, target, g, loss, saved, saved_bytes, ws, ws_bytes, s);
        if (rc != TFX_OK || (!dx && !dcoef)) return rc;
        return tfx_plan_backward(p, x, g, dx, dcoef, saved, saved_bytes, ws, ws_bytes, s);
    }
    // the arguments of both calls, checked before anything is enqueued
    const size_t need = std::max(p->ws_fused, p->bws_bytes);
    int rc = check_exec_args(p, x, y, ws, ws_bytes, need);
    if (rc != TFX_OK) return rc;
    if (x == y || !target || !g) return TFX_ERR_INVALID;
    const int64_t C = p->C, N = p->N;
    const size_t span = signal_span(C, N, p->ld);
    if (bytes_overlap(g, span, x, span) || bytes_overlap(g, span, y, span) ||
        (g != target && bytes_overlap(g, span, target, span)) || bytes_overlap(target, span, y, span) ||
        bytes_overlap(loss, sizeof(double), g, span) || bytes_overlap(loss, sizeof(double), y, span))
        return TFX_ERR_INVALID;
    if (dx && (ranges_overlap_not_equal(g, dx, C, N, p->ld) || bytes_overlap(x, span, dx, span)))
        return TFX_ERR_INVALID;
    if (bytes_overlap(dcoef, (size_t)p->ncoef * sizeof(double), g, span) ||
        bytes_overlap(dcoef, (size_t)p->ncoef * sizeof(double), y, span) ||
        bytes_overlap(loss, sizeof(double), dcoef, (size_t)p->ncoef * sizeof(double)))
        return TFX_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    const HostUnit& c = p->chain;
    const double inv = 1.0 / ((double)C * (double)N);
    if (cudaMemsetAsync(loss, 0, sizeof(double), st) != cudaSuccess) return TFX_ERR_CUDA;
    FirFftArgs f{};
    f.x = x;
    f.ldx = p->ld;
    f.y = y;
    f.ldy = p->ld;
    f.C = C;
    f.N = N;
    f.L = c.L;
    f.M = c.fft_M;
    f.m = c.fft_m;
    f.B = c.fft_B;
    f.P = 0;
    f.nbpc = c.ntt;
    f.nb = C * c.ntt;
    f.H = reinterpret_cast<const float2*>(p->dconst + c.off_H);
    f.tw = reinterpret_cast<const float2*>(p->dconst + c.off_tw);
    f.tgt = target;
    f.gout = g;
    f.loss = loss;
    f.gscale = (float)(2.0 * inv);
    f.lscale = inv;
    char* w = static_cast<char*>(ws);
    if (launch_fir_fft_train(f, reinterpret_cast<float2*>(w + p->b_sp_part), p->spec_grid, st) != cudaSuccess)
        return TFX_ERR_CUDA;
    return spectral_grads_from_partials(p, g, dx, dcoef, w, st, false, nullptr);
}

int tfx_plan_train_step_mse_launch_count(const tfx_plan* p, int with_dx, int with_dcoef) {
    if (!p || !p->train) return -1;
    if (p->C == 0 || p->N == 0) return 0;
    if (!(p->spectral && with_dcoef)) {
        const int b = (with_dx || with_dcoef) ? tfx_plan_backward_launch_count(p, with_dx, with_dcoef) : 0;
        return tfx_plan_forward_train_mse_launch_count(p) + b;
    }
    int n = 1;
    float dummy_dx;
    double dummy_dc;
    spectral_grads_from_partials(const_cast<tfx_plan*>(p), nullptr, with_dx ? &dummy_dx : nullptr, &dummy_dc, nullptr,
                                 nullptr, true, &n);
    return n;
}

int tfx_mse(const float* y, const float* target, float* g, int64_t C, int64_t N, int64_t ld, double* loss,
            tfx_stream s) {
    if (C < 0 || N < 0 || ld < (N > 1 ? N : 1) || !loss) return TFX_ERR_INVALID;
    if (C > 0 && N > 0 && (!y || !target)) return TFX_ERR_INVALID;
    return launch_mse(y, target, g, C, N, ld, loss, reinterpret_cast<cudaStream_t>(s)) == cudaSuccess ? TFX_OK
                                                                                          : TFX_ERR_CUDA;
}

size_t tfx_chain_workspace_size(int64_t C, int64_t N, int64_t ld, const tfx_stage* st, int32_t nst) {
    if (check_dims(C, N, ld) != TFX_OK || validate_stages(st, nst) != TFX_OK) return SIZE_MAX;
    tfx_plan p;  // layout only: nothing is allocated or uploaded
    p.C = C;
    p.N = N;
    p.ld = ld;
    if (build_plan(&p, st, nst, false) != TFX_OK) return SIZE_MAX;
    return p.ws_fused;
}

int tfx_chain(const float* x, float* y, int64_t C, int64_t N, int64_t ld, const tfx_stage* st, int32_t nst,
              void* ws, size_t ws_bytes, tfx_stream s) {
    int rc = check_dims(C, N, ld);
    if (rc != TFX_OK) return rc;
    rc = validate_stages(st, nst);
    if (rc != TFX_OK) return rc;
    if (C > 0 && N > 0 && (!x || !y)) return TFX_ERR_INVALID;
    if (ranges_overlap_not_equal(x, y, C, N, ld)) return TFX_ERR_INVALID;
    if (C == 0 || N == 0) return TFX_OK;
    CacheEntry e;
    rc = cached_plan(C, N, ld, st, nst, reinterpret_cast<cudaStream_t>(s), &e);
    if (rc != TFX_OK) return rc;
    if (ws) return tfx_plan_execute(e.plan, x, y, ws, ws_bytes, s);
    return tfx_plan_execute(e.plan, x, y, e.ws, e.ws_bytes, s);
}

int tfx_fir(const float* x, float* y, int64_t C, int64_t N, int64_t ld, const double* h, int32_t taps,
            tfx_stream s) {
    tfx_stage st = {TFX_STAGE_FIR, taps, h};
    return tfx_chain(x, y, C, N, ld, &st, 1, nullptr, 0, s);
}

int tfx_sos(const float* x, float* y, int64_t C, int64_t N, int64_t ld, const double* sos, int32_t sections,
            tfx_stream s) {
    tfx_stage st = {TFX_STAGE_SOS, sections, sos};
    return tfx_chain(x, y, C, N, ld, &st, 1, nullptr, 0, s);
}

void tfx_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_cache) free_entry(kv.second.first);
    g_cache.clear();
    g_lru.clear();
}

const char* tfx_strerror(int status) {
    switch (status) {
        case TFX_OK: return "TFX_OK";
        case TFX_ERR_INVALID: return "TFX_ERR_INVALID: invalid argument";
        case TFX_ERR_UNSTABLE: return "TFX_ERR_UNSTABLE: SOS section with a pole on or outside the unit circle";
        case TFX_ERR_WORKSPACE: return "TFX_ERR_WORKSPACE: workspace missing, too small or misaligned";
        case TFX_ERR_CUDA: return "TFX_ERR_CUDA: CUDA runtime call failed";
        case TFX_ERR_TIMEOUT: return "TFX_ERR_TIMEOUT: a device-side bounded wait gave up";
        case TFX_ERR_UNSUPPORTED: return "TFX_ERR_UNSUPPORTED: request outside what this build implements";
        case TFX_ERR_NOMEM: return "TFX_ERR_NOMEM: allocation failed";
        case TFX_ERR_DECAY: return "TFX_ERR_DECAY: the chain's response outlasts the spectral plan's overlap";
        default: return "unknown tfx status";
    }
}

int tfx_version(void) { return 0x000100; }

}  // extern "C"
