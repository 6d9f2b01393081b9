// tfx_sos_noalloc: the SOS-cascade scan for callers that must not allocate
// device memory (see include/tfx.h).  Everything the scan kernel needs beyond
// x and y -- its tile ticket, status word, look-back carries, and the
// per-section constants -- lives in one file-scope static device array of fixed
// size, so a call makes no cudaMalloc / cudaFree and uses no allocating
// library routine.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "plan_internal.cuh"

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

// Section constants of one call, passed to the set-up kernel by value (no
// host-to-device copy): the a0-normalised c-form coefficients in FP64.
struct NaSections {
    double b0[NA_MAX_SECTIONS], c1[NA_MAX_SECTIONS], c2[NA_MAX_SECTIONS], a1[NA_MAX_SECTIONS],
        a2[NA_MAX_SECTIONS];
};

// One CTA per section: its FP32 coefficients, and the chunk-transfer powers
// A^k (k < PW_LEN, A = M^T_CASCADE, M = [[-a1, 1], [-a2, 0]] the one-sample
// transfer of the c-form state) in FP64 by binary exponentiation, rounded
// once, written into the static array where the scan kernel reads them.
__global__ void k_noalloc_setup(NaSections sp, float* __restrict__ coef, float4* __restrict__ pw) {
    const int s = blockIdx.x;
    const double a1 = sp.a1[s], a2 = sp.a2[s];
    if (threadIdx.x == 0) {
        float* c = coef + 8 * s;
        c[0] = (float)sp.b0[s];
        c[1] = (float)sp.c1[s];
        c[2] = (float)sp.c2[s];
        c[3] = (float)a1;
        c[4] = (float)a2;
        c[5] = c[6] = c[7] = 0.f;
    }
    double m00 = -a1, m01 = 1.0, m10 = -a2, m11 = 0.0;
    double A00 = 1.0, A01 = 0.0, A10 = 0.0, A11 = 1.0;
    for (int e = T_CASCADE; e > 0; e >>= 1) {
        if (e & 1) {
            const double t00 = A00 * m00 + A01 * m10, t01 = A00 * m01 + A01 * m11;
            const double t10 = A10 * m00 + A11 * m10, t11 = A10 * m01 + A11 * m11;
            A00 = t00, A01 = t01, A10 = t10, A11 = t11;
        }
        const double q00 = m00 * m00 + m01 * m10, q01 = m00 * m01 + m01 * m11;
        const double q10 = m10 * m00 + m11 * m10, q11 = m10 * m01 + m11 * m11;
        m00 = q00, m01 = q01, m10 = q10, m11 = q11;
    }
    for (int k = threadIdx.x; k < PW_LEN; k += blockDim.x) {
        double p00 = 1.0, p01 = 0.0, p10 = 0.0, p11 = 1.0;
        double b00 = A00, b01 = A01, b10 = A10, b11 = A11;
        for (int e = k; e > 0; e >>= 1) {
            if (e & 1) {
                const double t00 = p00 * b00 + p01 * b10, t01 = p00 * b01 + p01 * b11;
                const double t10 = p10 * b00 + p11 * b10, t11 = p10 * b01 + p11 * b11;
                p00 = t00, p01 = t01, p10 = t10, p11 = t11;
            }
            const double q00 = b00 * b00 + b01 * b10, q01 = b00 * b01 + b01 * b11;
            const double q10 = b10 * b00 + b11 * b10, q11 = b10 * b01 + b11 * b11;
            b00 = q00, b01 = q01, b10 = q10, b11 = q11;
        }
        pw[(size_t)s * PW_LEN + k] = make_float4((float)p00, (float)p01, (float)p10, (float)p11);
    }
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

    // normalise and check every row on the host (FP64, a few doubles on the
    // stack); the device tables are built by a set-up kernel from these
    // values passed by value, so the call copies nothing from host memory
    NaSections sp{};
    for (int s = 0; s < sections; ++s) {
        const double* r = sos + 6 * s;
        for (int j = 0; j < 6; ++j)
            if (!std::isfinite(r[j])) return TFX_ERR_INVALID;
        if (r[3] == 0.0) return TFX_ERR_INVALID;
        const double b0 = r[0] / r[3], b1 = r[1] / r[3], b2 = r[2] / r[3], a1 = r[4] / r[3], a2 = r[5] / r[3];
        if (!(std::fabs(a2) < 1.0 && std::fabs(a1) < 1.0 + a2)) return TFX_ERR_UNSTABLE;
        // this entry point keeps FP32 cross-tile carries: a pole beyond the
        // radius where the plans switch to FP64 carries is not supported
        const double disc = a1 * a1 - 4.0 * a2;
        const double rad = disc < 0.0 ? std::sqrt(a2)
                                      : std::max(std::fabs(-a1 + std::sqrt(disc)), std::fabs(-a1 - std::sqrt(disc))) / 2.0;
        if (rad > HIQ_RADIUS) return TFX_ERR_UNSUPPORTED;
        sp.b0[s] = b0;
        sp.c1[s] = b1 - a1 * b0;
        sp.c2[s] = b2 - a2 * b0;
        sp.a1[s] = a1;
        sp.a2[s] = a2;
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
    k_noalloc_setup<<<sections, 256, 0, s>>>(sp, reinterpret_cast<float*>(base + NA_OFF_COEF),
                                             reinterpret_cast<float4*>(base + NA_OFF_PW));
    if (cudaGetLastError() != cudaSuccess) return TFX_ERR_CUDA;

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
