// labf_internal.cuh -- device-side data layout and helpers of the lambda-ABF
// engine.  Included by every translation unit of liblabf.
//
// Layout (all walkers of all systems in one arena, see labf_api.cu):
//   * Atoms of each walker live in "slots", grouped in super-clusters of 64
//     slots = 8 i-clusters of 8 = 16 j-clusters of 4, sorted spatially at
//     every neighbour-list rebuild (columns in xy, z order inside a column,
//     a 4-level k-d split inside each super-cluster).  Dummy slots pad the
//     last super-cluster of each column.
//   * Per slot: xq = (x, y, z, q sqrt(coul)), vv = (v, 0), xref = x at the
//     last rebuild, lj = (sigma/2, 2 sqrt(eps)), im = (1/m, sqrt(kT/m)),
//     F = 3 x int64 fixed point (2^-32 force units), uq = quantized
//     coordinates + atom id.
//   * Cluster-pair list: for each super-cluster, entries (j-cluster base
//     slot, periodic shift, mask of i-clusters) each with eight 32-bit
//     atom-pair masks (one bit per lane of an 8 i x 4 j warp tile).
//   * Alchemical list: per (walker, alchemical atom) the slots of its
//     environment atoms within the list radius.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "labf.h"

namespace labf {

constexpr int SC = 64;           // slots per super-cluster
constexpr int IC = 8;            // slots per i-cluster
constexpr int JC = 4;            // slots per j-cluster
constexpr int NIC = SC / IC;     // i-clusters per super-cluster
constexpr int NJC = SC / JC;     // j-clusters per super-cluster
constexpr int MAX_COL = 2048;    // atoms per column (sort kernel capacity)
constexpr int N_ETERMS = 8;      // LA_N_TERMS + spare
constexpr float FIX_TO_F = 2.3283064365386963e-10f;  // 2^-32
constexpr float F_TO_FIX = 4294967296.0f;            // 2^32
constexpr double E_TO_FIX = 16777216.0;              // 2^24 (energies)
constexpr float FIX_LIMIT = 1073741824.0f;           // 2^30: |F| beyond risks int64 overflow

struct SysDev {
    int n_atoms, atom_off;        // atoms; offset into per-system atom arrays
    int n_alch, alch_off;         // alchemical atoms; offset into alch_atoms
    int w_first, w_count;         // the system's walkers (consecutive)
    int P;                        // theta parameters: 3 n_alch + 1
    double box, box_inv;
    float boxf, box_invf;
    float rc2, krf, crf, sqrt_coul;
    double b_v, b_e;
    float sc_alpha;
    int sc_n, sc_m;
    float dt, c_at, s_at;         // atoms: dt, exp(-gamma dt), sqrt(1 - c^2)
    double dt_d, m_lambda, c_lm, sd_lm, kT;  // lambda particle
    float half_skin2;             // (skin / 2)^2
    float near_skin2;             // (NEAR_FRACTION skin / 2)^2: "due soon" for coalescing
    float prune_disp2;            // squared displacement that triggers pruning (0: off)
    float rprune2;                // (r_c + prune margin)^2
    long long R;                  // integer list threshold
    int Rq;                       // list radius in quantized units (rounded up)
    int ncx;                      // columns per dimension
    int cspan;                    // candidate columns per dimension around a super-cluster
    int bond_off, n_bonds, angle_off, n_angles, posres_off, n_posres;
    float posres_k;
    int fb_off, n_fb_a, n_fb_b;
    float fb_d0, fb_k;
    int lh_off, n_lh, lh_dims;
    double lh_k0, lh_k1;
    int lr_off, n_lr;             // lambda-dependent distance restraints
    double lr_delta, lr_k;
    uint32_t seed;
    int lambda_dynamics, abf_on, theta_stats, shared_freq;
    double n_full;
};

struct WalkerDev {
    int sys, stage, wlocal;       // system, stage (global), index within the system
    int slot_off, sc_cap;         // first global slot; super-cluster capacity
    int sc_off;                   // first global super-cluster
    int col_off, n_cols;          // columns
    int atom_base;                // first entry in per-walker atom arrays
    int alch_base;                // first (walker, alchemical atom) index
    int item_base, item_cap;      // pair-kernel work items
    int bo_off, n_bo;             // bonded work items (bonds, angles, posres)
};

struct StageDev {
    int sys, w0, w1, n_bins, bin_off;
    double lo, hi, width;
};

struct Dev {
    int n_sys, n_walkers, n_stages;
    int ent_cap;                  // entries per super-cluster
    int alch_cap;                 // environment atoms per alchemical atom
    int max_bins, P_max;
    int chunk;                    // entries per pair work item
    int total_bo;
    // array extents, for the range checks of debug builds (LA_CHECKS)
    int n_slots, n_scs, n_atoms_w, n_atoms_s, n_items_all;
    const SysDev *sys;
    const WalkerDev *walk;
    const StageDev *stage;
    // per-system atoms
    const float4 *ap;             // (q sqrt(coul), sigma/2, 2 sqrt(eps), 1/m)
    const float *anoise;          // sqrt(kT/m)
    const int *agroup;
    const int4 *aexcl;
    const unsigned char *aalch;
    const int *alch_atoms;        // per system: alchemical atom indices
    float4 *aparam_mut;           // mutable copy of ap (differentiation path)
    // topology
    const int2 *bond_ij;
    const float2 *bond_p;         // (r0, k)
    const int4 *angle_ijk;
    const float2 *angle_p;        // (theta0, k)
    const int *posres_idx;
    const float4 *posres_x0;
    const int *fb_idx;            // group a then group b
    const int *lh_idx;
    const float4 *lh_x0;
    const int2 *lr_ij;
    // per slot
    float4 *xq, *vv, *xref;
    float2 *lj, *im;
    int *atom_of_slot, *slot_walker;
    unsigned long long *F;
    int4 *uq;
    int2 *smeta;                  // per slot: (exclusion group, alchemical flag)
    int4 *sexcl;                  // per slot: extra excluded partners (atom ids)
    // rebuild scratch
    float4 *t_xq, *t_vv;
    int *t_old;
    int4 *t_uq;
    int *t_col, *t_pos, *bucket;
    // per walker atoms
    int *slot_of_atom;
    // columns and super-clusters
    int *col_count, *col_start, *col_sc, *col_nsc;
    int *n_sc;
    int *sc_member, *sc_n;
    int4 *bb_sc, *bb_ic, *bb_jc;  // (lo, hi) pairs; lo.w = real count
    int *sc_nent;
    int2 *ent_hdr;                // (j-cluster base global slot, shift bits | imask << 8)
    unsigned char *ent_lb;        // 32 per entry: lane l's bit ic = pair (8 ic + (l & 7), l >> 3)
    // per (super-cluster, candidate column) sub-lists written by the list
    // builder and compacted into ent_* in a fixed order
    int ncs, sub_cap;
    int2 *sub_hdr;
    unsigned char *sub_lb;
    int *sub_n;
    int4 *items;                  // (global sc, e0, e1, walker)
    int *n_items;
    // alchemical lists and partial sums
    int *alch_cnt, *alch_slot;
    double *alch_out;             // 4 per (walker, alch): dU/dlv, dU/dle, U_sc, le U_rf
    double *alch_th;              // 6 per (walker, alch): dU/d(eps, sig, q), d2 v(eps, sig), d2 e(q)
    // per walker
    double *lam, *plam, *G, *s, *dl_direct, *wth;
    unsigned long long *step;
    int *pending, *rebuild;
    long long *eterm;             // N_ETERMS per walker, 2^-24 fixed point
    // ABF
    double *abf_sum, *abf_sumsq;
    unsigned long long *abf_count;
    double *dl_sum, *dl_sumsq;
    unsigned long long *dl_count;
    double *th_d2, *th_d, *th_sd;
    // status and counters
    unsigned int *status;
    unsigned int *wdone, *sdone;  // arrivals per walker / per stage in the fused pair launch
    float4 *xprune;               // positions at the last pruning, per slot
    int *prune;                   // per walker: pruning requested (displacement or fresh list)
    int *near;                    // per walker: an atom of its system moved NEAR_FRACTION skin/2
    unsigned long long *prune_now;  // per walker: 0, or 1 + the step counter of the batched
                                    // step whose pair pass re-prunes the walker's tiles
    unsigned long long *counters; // [0] rebuilds [1] pairs normal [2] pairs alch [4, 5] pair
                                  // work items [6] rebuild events [8, 9] list-build work items
                                  // [10] re-pruning passes after a displacement trigger
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// Rebuild coalescing: a system whose atoms have moved NEAR_FRACTION of the
// rebuild threshold rebuilds together with any other system that must
// rebuild in the same step, so that batches of several systems share list
// builds instead of paying one chain of list kernels each.
constexpr float NEAR_FRACTION = 0.8f;

__device__ __forceinline__ void set_status(const Dev &d, unsigned bits) { atomicOr(d.status, bits); }

// Debug builds (nvcc -DLA_CHECKS=1; build(checks=True) in the package's
// build script) range-check every list, cell, slot and atom index read from
// device memory before it is used: a failed check sets LA_STATUS_BAD_INDEX
// and the caller skips the access (never a trap).  Release builds compile
// the checks away.
#ifndef LA_CHECKS
#define LA_CHECKS 0
#endif
__device__ __forceinline__ bool la_in(const Dev &d, long long i, long long n) {
    if (!LA_CHECKS) return true;
    if (i >= 0 && i < n) return true;
    set_status(d, LA_STATUS_BAD_INDEX);
    return false;
}

// a slot index read from a device array, checked in debug builds (a bad one
// becomes slot 0 once the status bit is set)
__device__ __forceinline__ int checked_slot(const Dev &d, int g) { return la_in(d, g, d.n_slots) ? g : 0; }

// round(f * 2^32) as a two's-complement int64, rounded to nearest (ties to
// even) and symmetric in sign, from FP32 arithmetic and 32-bit conversions
// only (a float -> int64 conversion instruction would run on the FP64 pipe,
// which is narrow on this GPU).  With a = |f|, h = floor(a) and r = a - h,
// r is exact (the fraction of a float is a float) and so is r 2^32 < 2^32;
// a 2^32 = h 2^32 + r 2^32 with h 2^32 an even integer, so rounding r 2^32
// once rounds a 2^32.  |f| is clamped below 2^31 (NaN maps to the clamp):
// a contribution that large, and any NaN, shows up as a summed force beyond
// the fixed-point range, which the integrator reports.
__device__ __forceinline__ unsigned long long f2fix(float f) {
    const float a = fminf(fabsf(f), 2147483520.0f);  // largest float below 2^31
    const float h = floorf(a);
    const unsigned hi = __float2uint_rz(h);
    const unsigned lo = __float2uint_rn((a - h) * 4294967296.0f);
    const unsigned long long v = ((unsigned long long)hi << 32) | lo;
    return f < 0.f ? (unsigned long long)(-(long long)v) : v;
}

// Fixed-point force accumulation (2^32 units per force unit).  Integer adds
// commute, so the sum is independent of the order of the atomics.
__device__ __forceinline__ void add_force(const Dev &d, int slot, float fx, float fy, float fz) {
    unsigned long long *p = d.F + 3 * (size_t)slot;
    atomicAdd(p + 0, f2fix(fx));
    atomicAdd(p + 1, f2fix(fy));
    atomicAdd(p + 2, f2fix(fz));
}

// fixed point back to float from its two 32-bit halves (no 64-bit
// conversion instruction): hi + lo 2^-32, within 1 ulp of the exact value
__device__ __forceinline__ float fix_to_float(unsigned long long v) {
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)(v & 0xffffffffull);
    return fmaf((float)lo, FIX_TO_F, (float)hi);
}

__device__ __forceinline__ float min_image(float dx, float L, float Linv) {
    return dx - L * rintf(dx * Linv);
}

// lambda -> (lambda_v, lambda_e) and slopes: linear to b_v / from b_e, flat
// beyond; slopes at the kinks taken on the flat side (Sec. 3.1.1).
__device__ __forceinline__ void lambda_path(double lam, double bv, double be, double &lv, double &le,
                                            double &dlv, double &dle) {
    if (lam < bv) {
        lv = lam / bv;
        dlv = 1.0 / bv;
    } else {
        lv = 1.0;
        dlv = 0.0;
    }
    if (lam > be) {
        le = (lam - be) / (1.0 - be);
        dle = 1.0 / (1.0 - be);
    } else {
        le = 0.0;
        dle = 0.0;
    }
}

// Philox4x32-10 (Salmon et al., SC'11): counter c, key k.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Four standard normals (Box-Muller on 24-bit uniforms) for counter
// {idx, step_lo, step_hi, tag} and key {seed, walker}.
__device__ __forceinline__ float4 normals4(uint32_t seed, uint32_t walker, unsigned long long step,
                                           uint32_t idx, uint32_t tag) {
    uint4 r = philox4x32_10(make_uint4(idx, (uint32_t)step, (uint32_t)(step >> 32), tag),
                            make_uint2(seed, walker));
    const float s24 = 5.9604644775390625e-08f;  // 2^-24
    float u1 = (float)((r.x >> 8) + 1u) * s24, u2 = (float)(r.y >> 8) * s24;
    float u3 = (float)((r.z >> 8) + 1u) * s24, u4 = (float)(r.w >> 8) * s24;
    float ra = sqrtf(-2.0f * logf(u1)), rb = sqrtf(-2.0f * logf(u3));
    float sa, ca, sb, cb;
    sincospif(2.0f * u2, &sa, &ca);
    sincospif(2.0f * u4, &sb, &cb);
    return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

// FP64 normal for the lambda particle (same stream definition, tag 1).
__device__ __forceinline__ double normal_lambda(uint32_t seed, uint32_t walker, unsigned long long step) {
    uint4 r = philox4x32_10(make_uint4(0u, (uint32_t)step, (uint32_t)(step >> 32), 1u),
                            make_uint2(seed, walker));
    const double s24 = 5.9604644775390625e-08;
    double u1 = (double)((r.x >> 8) + 1u) * s24, u2 = (double)(r.y >> 8) * s24;
    double sp, cp;
    sincospi(2.0 * u2, &sp, &cp);
    return sqrt(-2.0 * log(u1)) * cp;
}

// u = floor(frac(x L^-1) 2^24), one rounded FP64 product, no contraction.
__device__ __forceinline__ uint32_t quantize(float x, double box_inv) {
    double t = __dmul_rn((double)x, box_inv);
    double f = __dsub_rn(t, floor(t));
    double s = floor(__dmul_rn(f, 16777216.0));
    uint32_t q = (uint32_t)s;
    return q >= 16777216u ? 0u : q;
}

// minimum-image difference on the 2^24 torus, in [-2^23, 2^23)
__device__ __forceinline__ int torus_delta(int a, int b) { return ((a - b + 8388608) & 16777215) - 8388608; }

__device__ __forceinline__ int bin_of(double lam, const StageDev &st) {
    int k = (int)floor((lam - st.lo) / st.width);
    return k < 0 ? 0 : (k >= st.n_bins ? st.n_bins - 1 : k);
}

// warp-wide FP64 sum with a fixed shuffle tree (deterministic)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace labf
