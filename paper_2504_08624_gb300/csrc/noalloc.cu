// tfx_sos_noalloc: the SOS-cascade scan for callers that must not allocate
// device memory (see include/tfx.h).  Everything the scan kernel needs beyond
// x and y -- its tile ticket, status word, look-back carries, and the
// per-section constants -- lives in one file-scope static device array of fixed
// size, so a call makes no cudaMalloc / cudaFree and uses no allocating
// library routine.
#include <cmath>
#include <mutex>

#include "tfx_common.cuh"

namespace tfx {
namespace {

constexpr int NA_MAX_SECTIONS = 8;
constexpr int64_t NA_MAX_TILES = 32768;  // C * ceil(N / 8192)

// Layout of the static array (byte offsets).
constexpr size_t NA_OFF_TICKET = 0;
constexpr size_t NA_OFF_STATUS = 128;
constexpr size_t NA_OFF_CARRY = 256;
constexpr size_t NA_CARRY_BYTES = (size_t)NA_MAX_TILES * NA_MAX_SECTIONS * sizeof(Carry);
constexpr size_t NA_OFF_COEF = NA_OFF_CARRY + NA_CARRY_BYTES;
constexpr size_t NA_COEF_BYTES = (size_t)NA_MAX_SECTIONS * 8 * sizeof(float);
constexpr size_t NA_OFF_PW = NA_OFF_COEF + NA_COEF_BYTES;
constexpr size_t NA_PW_BYTES = (size_t)NA_MAX_SECTIONS * PW_LEN * sizeof(float4);
constexpr size_t NA_BYTES = NA_OFF_PW + NA_PW_BYTES;  // about 4.3 MB

constexpr int NA_MAX_DEVICES = 64;

}  // namespace
}  // namespace tfx

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_tfx_noalloc_scratch[tfx::NA_BYTES];

namespace tfx {
namespace {

std::mutex g_na_mu;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the static array for the current device, looked up once
// per device (host code must not use the symbol itself as a device pointer).
int na_scratch(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TFX_ERR_CUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return TFX_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_tfx_noalloc_scratch) != cudaSuccess || !p) return TFX_ERR_CUDA;
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_na_ptr[dev];
    return TFX_OK;
}

struct NaM2 {
    double a, b, c, d;
};
inline NaM2 na_mul(const NaM2& x, const NaM2& y) {
    return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}

}  // namespace
}  // namespace tfx

using namespace tfx;

extern "C" int tfx_sos_noalloc(const float* x, float* y, int64_t C, int64_t N, int64_t ld, const double* sos,
                               int32_t sections, tfx_stream stream) {
    if (C < 0 || N < 0 || ld < (N > 1 ? N : 1)) return TFX_ERR_INVALID;
    if (sections < 0 || (sections > 0 && !sos)) return TFX_ERR_INVALID;
    if (C == 0 || N == 0) return TFX_OK;
    if (!x || !y) return TFX_ERR_INVALID;
    if (x != y) {
        const char* xb = reinterpret_cast<const char*>(x);
        const char* yb = reinterpret_cast<const char*>(y);
        const size_t span = ((size_t)(C - 1) * (size_t)ld + (size_t)N) * sizeof(float);
        if (xb < yb + span && yb < xb + span) return TFX_ERR_INVALID;
    }
    if (sections > NA_MAX_SECTIONS) return TFX_ERR_UNSUPPORTED;
    const int64_t ntt = (N + TILE - 1) / TILE;
    if (C > NA_MAX_TILES / ntt) return TFX_ERR_UNSUPPORTED;

    // section constants, computed in FP64 on the stack (no heap use)
    float coef[NA_MAX_SECTIONS * 8] = {};
    float4 pw[NA_MAX_SECTIONS * PW_LEN];
    for (int s = 0; s < sections; ++s) {
        const double* r = sos + 6 * s;
        for (int j = 0; j < 6; ++j)
            if (!std::isfinite(r[j])) return TFX_ERR_INVALID;
        if (r[3] == 0.0) return TFX_ERR_INVALID;
        const double b0 = r[0] / r[3], b1 = r[1] / r[3], b2 = r[2] / r[3], a1 = r[4] / r[3], a2 = r[5] / r[3];
        if (!(std::fabs(a2) < 1.0 && std::fabs(a1) < 1.0 + a2)) return TFX_ERR_UNSTABLE;
        coef[8 * s + 0] = (float)b0;
        coef[8 * s + 1] = (float)(b1 - a1 * b0);
        coef[8 * s + 2] = (float)(b2 - a2 * b0);
        coef[8 * s + 3] = (float)a1;
        coef[8 * s + 4] = (float)a2;
        const NaM2 m = {-a1, 1.0, -a2, 0.0};
        NaM2 A = {1, 0, 0, 1};
        for (int t = 0; t < T_CASCADE; ++t) A = na_mul(A, m);  // samples per thread of the cascade kernel
        NaM2 pk = {1, 0, 0, 1};
        for (int k = 0; k < PW_LEN; ++k) {
            pw[s * PW_LEN + k] = make_float4((float)pk.a, (float)pk.b, (float)pk.c, (float)pk.d);
            pk = na_mul(pk, A);
        }
    }

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (sections == 0) return launch_copy_rows(x, y, C, N, ld, ld, s) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;

    unsigned char* base = nullptr;
    int rc = na_scratch(&base);
    if (rc != TFX_OK) return rc;
    const int64_t tiles = C * ntt;
    // ticket, status word and look-back carries must start at zero
    if (cudaMemsetAsync(base, 0, NA_OFF_CARRY + (size_t)tiles * sections * sizeof(Carry), s) != cudaSuccess)
        return TFX_ERR_CUDA;
    if (cudaMemcpyAsync(base + NA_OFF_COEF, coef, (size_t)sections * 8 * sizeof(float), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return TFX_ERR_CUDA;
    if (cudaMemcpyAsync(base + NA_OFF_PW, pw, (size_t)sections * PW_LEN * sizeof(float4),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TFX_ERR_CUDA;

    UnitArgs a{};
    a.x = x;
    a.y = y;
    a.ldx = ld;
    a.ldy = ld;
    a.C = C;
    a.N = N;
    a.ntt = ntt;
    a.k.S = sections;
    a.k.L = 0;
    a.k.H = 0;
    a.k.nkb = 0;
    a.k.gain = 1.0f;
    a.k.coef = reinterpret_cast<const float*>(base + NA_OFF_COEF);
    a.k.pw = reinterpret_cast<const float4*>(base + NA_OFF_PW);
    a.k.taps = nullptr;
    a.sc.ticket = reinterpret_cast<unsigned*>(base + NA_OFF_TICKET);
    a.sc.flags = nullptr;  // no FIR: no tails to flag
    a.sc.carry = reinterpret_cast<Carry*>(base + NA_OFF_CARRY);
    a.sc.tails = nullptr;
    a.sc.tail_len = 0;
    a.status = reinterpret_cast<int*>(base + NA_OFF_STATUS);
    a.drop_tile = -1;
    return launch_unit(a, s) == cudaSuccess ? TFX_OK : TFX_ERR_CUDA;
}
