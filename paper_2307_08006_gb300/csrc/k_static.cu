// k_static.cu -- la_alch_pairs_static: the alchemical part of the pair pass
// with its scratch in a file-scope static device array, for callers that
// cannot allocate device memory (a plugin inside a program that owns the
// GPU memory, or a deployment with a fixed device footprint).
//
// The scratch holds 64-bit fixed-point force accumulators (so the summed
// forces do not depend on the order of the atomics), per-alchemical-atom
// FP64 partial sums that are folded in a fixed order, and one status word
// (LA_STATUS_* bits: a bad alchemical index, a non-finite distance or force,
// a force beyond the fixed-point range), reported in out[5].  Every call
// clears the part it uses first.  All calls on a device share the array: calls whose
// GPU work overlaps race, so callers must serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "labf_internal.cuh"

// int64 force accumulators, then double partial sums, then the status word
#define LA_STATIC_FORCE_WORDS (3ull * LA_STATIC_MAX_ATOMS)
#define LA_STATIC_PART_WORDS (4ull * LA_STATIC_MAX_ALCH)
#define LA_STATIC_STATUS_WORDS 1ull

// The scratch array (about 3.2 MB on every device that loads the library).
// Host code must not take its address directly: the name is a host-side
// stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char
    g_static_scratch[8 * (LA_STATIC_FORCE_WORDS + LA_STATIC_PART_WORDS + LA_STATIC_STATUS_WORDS)];

namespace labf {
namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[MAX_DEVICES] = {nullptr};
thread_local std::string g_static_err;

struct StaticParams {
    int n, n_alch;
    float L, Linv, rc2, krf, crf, sqrt_coul;
    float le, lvn, dlvn, sa, dsdl;
};

__global__ void k_static_clear(unsigned long long *F, double *part, unsigned *status, int n, int n_alch) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x) F[i] = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * n_alch; i += gridDim.x * blockDim.x)
        part[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0u;
}

// a force component that fits the 64-bit fixed-point range, else a status bit
__device__ __forceinline__ bool static_force_ok(float fx, float fy, float fz, unsigned *status) {
    const float m = fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz)));
    if (m < FIX_LIMIT) return true;
    atomicOr(status, m == m ? LA_STATUS_FIXED_OVERFLOW : LA_STATUS_NONFINITE);
    return false;
}

// one warp per alchemical atom; lanes stride over all atoms
__global__ void k_static_alch(StaticParams p, const float *x, const float *q, const float *sig,
                              const float *eps, const uint8_t *alch, const int *grp, const int *alch_idx,
                              unsigned long long *F, double *part, unsigned *status) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= p.n_alch) return;
    const int a = alch_idx[r];
    if ((unsigned)a >= (unsigned)p.n || !alch[a]) {  // not an alchemical atom of this system
        if (lane == 0) atomicOr(status, LA_STATUS_BAD_INDEX);
        return;
    }
    const float xa = x[3 * a], ya = x[3 * a + 1], za = x[3 * a + 2];
    const float qa = q[a] * p.sqrt_coul, sa_half = 0.5f * sig[a], ea2 = 2.0f * sqrtf(fmaxf(eps[a], 0.f));
    const int ga = grp[a];
    float fax = 0.f, fay = 0.f, faz = 0.f;
    double sv = 0.0, se = 0.0, usc_s = 0.0, urf_s = 0.0;
    for (int b = lane; b < p.n; b += 32) {
        if (b == a || alch[b] || (ga >= 0 && grp[b] == ga)) continue;
        const float dx = min_image(xa - x[3 * b], p.L, p.Linv);
        const float dy = min_image(ya - x[3 * b + 1], p.L, p.Linv);
        const float dz = min_image(za - x[3 * b + 2], p.L, p.Linv);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < p.rc2)) {
            if (r2 != r2) atomicOr(status, LA_STATUS_NONFINITE);
            continue;
        }
        const float rinv = rsqrtf(r2);
        const float r2inv = rinv * rinv;
        const float qq = qa * q[b] * p.sqrt_coul;
        const float rf_u = qq * (rinv + p.krf * r2 - p.crf);
        const float rf_f = qq * (rinv * r2inv - 2.0f * p.krf);
        const float sg = sa_half + 0.5f * sig[b];
        const float e4 = ea2 * 2.0f * sqrtf(fmaxf(eps[b], 0.f));
        float sc_f = 0.f, usc = 0.f, dsc = 0.f;
        if (e4 > 0.f) {
            const float q2 = r2 / (sg * sg);
            const float rho6 = q2 * q2 * q2;
            const float is = 1.0f / (p.sa + rho6);
            const float g = is * is - is;
            const float g1 = is * is - 2.0f * is * is * is;
            usc = p.lvn * e4 * g;
            sc_f = -p.lvn * e4 * g1 * 6.0f * rho6 * r2inv;
            dsc = p.dlvn * e4 * g + p.lvn * e4 * g1 * p.dsdl;
        }
        const float fs = sc_f + p.le * rf_f;
        if (!static_force_ok(fs * dx, fs * dy, fs * dz, status)) continue;
        fax = fmaf(fs, dx, fax);
        fay = fmaf(fs, dy, fay);
        faz = fmaf(fs, dz, faz);
        atomicAdd(F + 3 * (size_t)b, (unsigned long long)__float2ll_rn(-fs * dx * F_TO_FIX));
        atomicAdd(F + 3 * (size_t)b + 1, (unsigned long long)__float2ll_rn(-fs * dy * F_TO_FIX));
        atomicAdd(F + 3 * (size_t)b + 2, (unsigned long long)__float2ll_rn(-fs * dz * F_TO_FIX));
        sv += (double)dsc;
        se += (double)rf_u;
        usc_s += (double)usc;
        urf_s += (double)(p.le * rf_u);
    }
    fax = warp_sumf(fax);
    fay = warp_sumf(fay);
    faz = warp_sumf(faz);
    sv = warp_sum(sv);
    se = warp_sum(se);
    usc_s = warp_sum(usc_s);
    urf_s = warp_sum(urf_s);
    if (lane == 0) {
        if (static_force_ok(fax, fay, faz, status)) {
            atomicAdd(F + 3 * (size_t)a, (unsigned long long)__float2ll_rn(fax * F_TO_FIX));
            atomicAdd(F + 3 * (size_t)a + 1, (unsigned long long)__float2ll_rn(fay * F_TO_FIX));
            atomicAdd(F + 3 * (size_t)a + 2, (unsigned long long)__float2ll_rn(faz * F_TO_FIX));
        }
        part[4 * r] = sv;
        part[4 * r + 1] = se;
        part[4 * r + 2] = usc_s;
        part[4 * r + 3] = urf_s;
    }
}

// forces out in FP32; partial sums folded in alchemical-atom order; status
__global__ void k_static_out(const unsigned long long *F, const double *part, const unsigned *status, int n,
                             int n_alch, double dlv, double dle, float *forces, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x)
        forces[i] = fix_to_float(F[i]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double sv = 0.0, se = 0.0, usc = 0.0, urf = 0.0;
        for (int r = 0; r < n_alch; ++r) {
            sv += part[4 * r];
            se += part[4 * r + 1];
            usc += part[4 * r + 2];
            urf += part[4 * r + 3];
        }
        out[0] = dlv * sv + dle * se;
        out[1] = sv;
        out[2] = se;
        out[3] = usc;
        out[4] = urf;
        out[5] = (double)*status;
    }
}

int static_fail(int code, const char *msg) {
    g_static_err = msg;
    return code;
}

// once per device, with that device current: the array's device address
int static_scratch(void **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(LA_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return static_fail(LA_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            char buf[256];
            snprintf(buf, sizeof buf, "cudaGetSymbolAddress of the static scratch failed: %s",
                     cudaGetErrorString(e));
            return static_fail(LA_ERR_CUDA, buf);
        }
        g_scratch_addr[dev] = p;
    }
    *ptr = g_scratch_addr[dev];
    return LA_OK;
}

}  // namespace
}  // namespace labf

using namespace labf;

extern "C" int la_alch_pairs_static(int n_atoms, const float *x, const float *q, const float *sigma,
                                    const float *epsilon, const uint8_t *alch, const int32_t *excl_group,
                                    int n_alch, const int32_t *alch_idx, double box, double r_cut,
                                    double eps_rf, double coul, double lam, double b_v, double b_e,
                                    double sc_alpha, int sc_n, int sc_m, float *forces, double *out,
                                    void *stream) {
    if (n_atoms <= 0 || n_alch < 0 || !x || !q || !sigma || !epsilon || !alch || !excl_group || !forces ||
        !out || (n_alch > 0 && !alch_idx))
        return static_fail(LA_ERR_INVALID_ARG, "NULL pointer or non-positive atom count");
    if (n_atoms > LA_STATIC_MAX_ATOMS || n_alch > LA_STATIC_MAX_ALCH) {
        char buf[160];
        snprintf(buf, sizeof buf, "size beyond the static scratch: n_atoms %d (max %d), n_alch %d (max %d)",
                 n_atoms, LA_STATIC_MAX_ATOMS, n_alch, LA_STATIC_MAX_ALCH);
        return static_fail(LA_ERR_INVALID_ARG, buf);
    }
    if (!(box > 0) || !(r_cut > 0) || 2.0 * r_cut > box || !(b_v > 0) || !(b_e < 1))
        return static_fail(LA_ERR_INVALID_ARG, "invalid box, cutoff or alchemical parameters");
    if (sc_n < 1 || sc_m < 1)  // n lambda_v^(n-1) and m (1-lambda_v)^(m-1) at the ends need n, m >= 1
        return static_fail(LA_ERR_INVALID_ARG, "soft-core powers sc_n and sc_m must be >= 1");
    void *base = nullptr;
    int rc = static_scratch(&base);
    if (rc != LA_OK) return rc;
    unsigned long long *F = (unsigned long long *)base;
    double *part = (double *)(F + LA_STATIC_FORCE_WORDS);
    unsigned *status = (unsigned *)(part + LA_STATIC_PART_WORDS);

    double lv, le, dlv, dle;
    if (lam < b_v) { lv = lam / b_v; dlv = 1.0 / b_v; } else { lv = 1.0; dlv = 0.0; }
    if (lam > b_e) { le = (lam - b_e) / (1.0 - b_e); dle = 1.0 / (1.0 - b_e); } else { le = 0.0; dle = 0.0; }
    StaticParams p;
    p.n = n_atoms;
    p.n_alch = n_alch;
    p.L = (float)box;
    p.Linv = (float)(1.0 / box);
    p.rc2 = (float)(r_cut * r_cut);
    const double krf = eps_rf <= 0.0 ? 1.0 / (2.0 * r_cut * r_cut * r_cut)
                                     : (eps_rf - 1.0) / ((2.0 * eps_rf + 1.0) * r_cut * r_cut * r_cut);
    p.krf = (float)krf;
    p.crf = (float)(1.0 / r_cut + krf * r_cut * r_cut);
    p.sqrt_coul = (float)std::sqrt(coul > 0.0 ? coul : 0.0);
    p.le = (float)le;
    p.lvn = (float)std::pow(lv, (double)sc_n);
    p.dlvn = (float)((double)sc_n * std::pow(lv, (double)(sc_n - 1)));
    p.sa = (float)(sc_alpha * std::pow(1.0 - lv, (double)sc_m));
    p.dsdl = (float)(-(double)sc_m * sc_alpha * std::pow(1.0 - lv, (double)(sc_m - 1)));

    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (3 * n_atoms + 255) / 256;
    k_static_clear<<<nb < 1024 ? nb : 1024, 256, 0, s>>>(F, part, status, n_atoms, n_alch);
    if (n_alch > 0) k_static_alch<<<(n_alch + 3) / 4, 128, 0, s>>>(p, x, q, sigma, epsilon, alch, excl_group,
                                                                    alch_idx, F, part, status);
    k_static_out<<<nb < 1024 ? nb : 1024, 256, 0, s>>>(F, part, status, n_atoms, n_alch, dlv, dle, forces, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(LA_ERR_CUDA, cudaGetErrorString(e));
    return LA_OK;
}

extern "C" const char *la_static_last_error(void) { return g_static_err.c_str(); }
