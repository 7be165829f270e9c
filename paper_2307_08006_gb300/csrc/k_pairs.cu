// k_pairs.cu -- the pair pass: LJ + reaction-field forces of normal pairs
// over the cluster-pair list, and, in the same launch, the alchemically
// scaled pairs with the walker's dU/dlambda partials (Sec. 3.1.2, Eq.
// lambda-abf: the engine provides dV/dlambda every step).
//
// Normal pairs: warps take work items (a chunk of one super-cluster's
// j-list) from a global counter.  The super-cluster's 64 slots sit in shared
// memory.  Entries are prepared 32 at a time, one per lane (header, periodic
// shift applied to the 4 j-atoms, lane mask bytes), into shared memory; then
// for each entry lane (ia, jb) = (lane & 7, lane >> 3) evaluates the pair
// (i-atom ia of every flagged i-cluster, j-atom jb).  One j-cluster load and
// one j-force reduction serve up to 8 x 32 pairs, and the eight i-force
// accumulators stay in registers for the whole item.  Forces are summed in
// FP32 and added to the 64-bit fixed-point force array with integer atomics
// (order-free, so results are bit-reproducible).  The i-forces are flushed
// to the fixed-point array after every 32 entries of a super-cluster's list,
// so every kernel variant and work-item size (a multiple of 32 entries)
// produces the same bits.  All float-to-fixed conversions use integer
// instructions: the hardware conversion to 64-bit integers runs on the FP64
// pipe, which is narrow on this GPU.
//
// Per in-cutoff pair (force only), 37 FP32 flops (FMA = 2) plus one rsqrt:
//   d = x_i - x_j (3), r2 (5), 1/r2 (1), sigma_ij = s_i + s_j, (sigma/r)^2,
//   (sigma/r)^6 (5), 4 eps_ij (sigma/r)^6 (2), t = 12 (sigma/r)^6 - 6 (2),
//   b = q_i q_j / r + 4eps (sigma/r)^6 t (4), f = b / r2 - 2 k_rf q_i q_j (3),
//   f_i += f d, f_j -= f d (12).
//
// Alchemical pairs: one warp per (walker, alchemical atom); lanes stride over
// its environment list.  Soft-core LJ lambda_v^n 4 eps (s^-2 - s^-1) with
// s = alpha (1 - lambda_v)^m + (r/sigma)^6, RF scaled by lambda_e; per-lane
// FP64 sums of dU/dlambda_v, dU/dlambda_e, energies and theta derivatives,
// reduced with a fixed shuffle tree (deterministic).
#include "labf_dyn.cuh"
#include "labf_internal.cuh"
#include "labf_launch.h"

namespace labf {

constexpr int EPC = 32;  // entries prepared per pass (one per lane)

// x^n for an integer n >= 0 (square and multiply; exact for n <= 1)
__device__ __forceinline__ double ipow(double x, int n) {
    double r = 1.0;
    for (; n > 0; n >>= 1) {
        if (n & 1) r *= x;
        x *= x;
    }
    return r;
}
constexpr unsigned FULL = 0xffffffffu;

template <int WARPS>
struct PairShared {
    float4 sxq[WARPS][SC];      // the item's super-cluster
    float2 slj[WARPS][SC];
    float4 jx[WARPS][EPC][JC];  // prepared j-atoms (shift applied)
    float2 jl[WARPS][EPC][JC];
    unsigned char lb[WARPS][EPC][32];
    int pre[LA_MAX_WALKERS_PER_LAUNCH + 1];
};

// counters[4] hands out work items; counters[5] counts warps that found no
// more work; the last one resets both for the next launch
constexpr int CTR_ITEM = 4, CTR_DONE = 5;

// i-forces of one flush, summed over the 4 j-lanes of each i-atom with a
// transposed tree: at the first level (partner jb ^ 1) a lane keeps the
// i-clusters {0, 1, 4, 5} (jb even) or {2, 3, 6, 7} (jb odd) and sends the
// others; at the second (partner jb ^ 2) it keeps the lower or upper pair, so
// lane (ia, jb) ends with i-clusters 2jb and 2jb + 1.  Every i-atom's sum is
// (a0 + a1) + (a2 + a3) over the j-lanes.  The accumulators restart from zero.
__device__ __forceinline__ void flush_i(const Dev &d, int gS, int ia, int jb, unsigned touched,
                                        float (&fi)[NIC][3]) {
    const bool odd = (jb & 1) != 0, upper = (jb & 2) != 0;
    float k1[4][3];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int ke = t < 2 ? t : t + 2;  // 0, 1, 4, 5
        const int ko = ke + 2;             // 2, 3, 6, 7
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float keep = odd ? fi[ko][c] : fi[ke][c];
            const float send = odd ? fi[ke][c] : fi[ko][c];
            k1[t][c] = keep + __shfl_xor_sync(FULL, send, 8);
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int ic = 2 * jb + t;
        unsigned long long *p = d.F + 3 * (size_t)(gS + ic * IC + ia);
        const bool on = (touched >> ic) & 1u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float keep = upper ? k1[t + 2][c] : k1[t][c];
            const float send = upper ? k1[t][c] : k1[t + 2][c];
            const float v = keep + __shfl_xor_sync(FULL, send, 16);
            if (on) atomicAdd(p + c, f2fix(v));
        }
    }
#pragma unroll
    for (int ic = 0; ic < NIC; ++ic) fi[ic][0] = fi[ic][1] = fi[ic][2] = 0.f;
}

// j-forces of two entries A and B at once (B absent: pass zeros and
// has_b = false).  Lane (ia, jb) holds j-atom jb's partial sums over its
// i-atoms (a for A, b for B; positive accumulation, the atom receives minus
// the sum).  Transposed tree over the 8 i-lanes: partner ia ^ 4 (lanes
// ia < 4 keep A, the others B), ia ^ 2 (keep x, y or z, 0), ia ^ 1; lane ia
// ends with A's component ia (ia < 3) or B's component ia - 4 (4 <= ia < 7).
// Each sum is ((a0 + a4) + (a2 + a6)) + ((a1 + a5) + (a3 + a7)), whether or
// not B is present.
__device__ __forceinline__ void flush_j2(const Dev &d, int gjA, int gjB, bool has_b, int ia, const float (&a)[3],
                                         const float (&b)[3]) {
    const bool h4 = (ia & 4) != 0, h2 = (ia & 2) != 0, h1 = (ia & 1) != 0;
    float v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float keep = h4 ? b[c] : a[c];
        const float send = h4 ? a[c] : b[c];
        v[c] = keep + __shfl_xor_sync(FULL, send, 4);
    }
    // (x, y) kept by h2 = 0, (z, 0) by h2 = 1
    const float k0 = h2 ? v[2] : v[0], k1 = h2 ? 0.f : v[1];
    const float s0 = h2 ? v[0] : v[2], s1 = h2 ? v[1] : 0.f;
    const float w0 = k0 + __shfl_xor_sync(FULL, s0, 2);
    const float w1 = k1 + __shfl_xor_sync(FULL, s1, 2);
    const float kk = h1 ? w1 : w0, ss = h1 ? w0 : w1;
    const float c = kk + __shfl_xor_sync(FULL, ss, 1);
    const int comp = ia & 3;
    if (comp < 3 && (!h4 || has_b)) atomicAdd(d.F + 3 * (size_t)(h4 ? gjB : gjA) + comp, f2fix(-c));
}

// One work item's entries, prepared and evaluated 32 at a time; the
// i-forces are flushed after every 32 entries.  MSHIFT: 8 reads the i-cluster
// mask pruned for the batched step, 16 the listed one (one-task launches,
// which run without pruning).  PRUNE (batched step, walker due for
// re-pruning): the listed mask is evaluated and each entry's pruned mask is
// rewritten with the i-clusters holding a listed pair within r_c + margin (a
// ballot per tile), which later steps read; every tile that is skipped adds
// exact zeros, so results do not depend on the pruning.
template <bool ENERGY, int WARPS, int MSHIFT, bool PRUNE>
__device__ __forceinline__ void item_entries(const Dev &d, PairShared<WARPS> &sh, const SysDev &S, int4 it, int gS,
                                             float &elj, float &erf, int &npair) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int ia = lane & 7, jb = lane >> 3;
    const float L = S.boxf, rc2 = S.rc2, krf2 = 2.0f * S.krf, krf = S.krf, crf = S.crf;
    const float rp2 = S.rprune2;
    float fi[NIC][3];
#pragma unroll
    for (int ic = 0; ic < NIC; ++ic) fi[ic][0] = fi[ic][1] = fi[ic][2] = 0.f;
    unsigned touched = 0;
    const size_t ebase = (size_t)it.x * d.ent_cap;
    for (int eb = it.y; eb < it.z; eb += EPC) {
        const int ne = min(EPC, it.z - eb);
        // prepare up to 32 entries, one per lane
        int gj_l = 0, hy_l = 0;
        unsigned im_l = 0, keep_l = 0;
        __syncwarp();
        if (lane < ne) {
            const int2 hdr = d.ent_hdr[ebase + eb + lane];
            gj_l = hdr.x;
            hy_l = hdr.y;
            im_l = ((unsigned)hdr.y >> (PRUNE ? 16 : MSHIFT)) & 0xffu;
            if (!la_in(d, gj_l, d.n_slots - JC + 1)) gj_l = 0, im_l = 0;  // entry skipped
            const float sx = (float)((hdr.y & 3) - 1) * L;
            const float sy = (float)(((hdr.y >> 2) & 3) - 1) * L;
            const float sz = (float)(((hdr.y >> 4) & 3) - 1) * L;
#pragma unroll
            for (int q = 0; q < JC; ++q) {
                float4 x = d.xq[gj_l + q];
                x.x += sx;
                x.y += sy;
                x.z += sz;
                sh.jx[wib][lane][q] = x;
                sh.jl[wib][lane][q] = d.lj[gj_l + q];
            }
            const uint4 *src = reinterpret_cast<const uint4 *>(d.ent_lb + 32 * (ebase + eb + lane));
            uint4 *dst = reinterpret_cast<uint4 *>(&sh.lb[wib][lane][0]);
            dst[0] = src[0];
            dst[1] = src[1];
        }
        // entries whose tiles were all pruned add nothing: skip them
        unsigned emask = __ballot_sync(FULL, im_l != 0u);
        __syncwarp();
        // one entry: every flagged i-cluster against the entry's j-cluster;
        // fjs receives j-atom jb's partial force over this lane's i-atoms.
        // The re-pruning form evaluates every listed tile: the atom whose
        // displacement triggered it may already have moved past the margin
        // the previous pruning allowed for.
        auto entry = [&](int k, float (&fjs)[3]) {
            const unsigned imask = __shfl_sync(FULL, im_l, k);
            const float4 xj = sh.jx[wib][k][jb];
            const float2 lj_j = sh.jl[wib][k][jb];
            const unsigned lb = sh.lb[wib][k][lane];
            touched |= imask;
            float fj[3] = {0.f, 0.f, 0.f};
            unsigned kb = 0;  // this lane's pairs within r_c + margin, per i-cluster
#pragma unroll
            for (int ic = 0; ic < NIC; ++ic) {
                if (imask & (1u << ic)) {
                    const float4 xi = sh.sxq[wib][ic * IC + ia];
                    const float2 li = sh.slj[wib][ic * IC + ia];
                    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (PRUNE) kb |= ((lb & (1u << ic)) && r2 < rp2) ? 1u << ic : 0u;
                    const bool in = (lb & (1u << ic)) && (r2 < rc2);
                    const float rinv = rsqrtf(r2);
                    const float r2inv = rinv * rinv;
                    const float sg = li.x + lj_j.x;
                    const float sr2 = sg * sg * r2inv;
                    const float sr6 = sr2 * sr2 * sr2;
                    const float e4s6 = li.y * lj_j.y * sr6;
                    const float qq = xi.w * xj.w;
                    const float b = fmaf(qq, rinv, e4s6 * fmaf(12.f, sr6, -6.f));
                    float fs = fmaf(b, r2inv, -qq * krf2);
                    fs = in ? fs : 0.f;
                    fi[ic][0] = fmaf(fs, dx, fi[ic][0]);
                    fi[ic][1] = fmaf(fs, dy, fi[ic][1]);
                    fi[ic][2] = fmaf(fs, dz, fi[ic][2]);
                    fj[0] = fmaf(fs, dx, fj[0]);
                    fj[1] = fmaf(fs, dy, fj[1]);
                    fj[2] = fmaf(fs, dz, fj[2]);
                    if (ENERGY) {
                        if (in) {
                            elj += e4s6 * (sr6 - 1.f);
                            erf += qq * (rinv + krf * r2 - crf);
                            ++npair;
                        }
                    }
                }
            }
            if (PRUNE) {
                const unsigned keep = __reduce_or_sync(FULL, kb);
                keep_l = lane == k ? keep : keep_l;
            }
            fjs[0] = fj[0];
            fjs[1] = fj[1];
            fjs[2] = fj[2];
        };
        // two entries per iteration (also in the re-pruning form): the
        // compiler interleaves their independent loads and arithmetic (the
        // order of every sum stays), and one transposed reduction serves both
        // j-clusters
        while (emask) {
            const int k0 = __ffs(emask) - 1;
            emask &= emask - 1u;
            float a[3], b[3] = {0.f, 0.f, 0.f};
            const int gA = __shfl_sync(FULL, gj_l, k0) + jb;
            int gB = 0;
            const bool two = emask != 0u;
            if (two) {
                const int k1 = __ffs(emask) - 1;
                emask &= emask - 1u;
                gB = __shfl_sync(FULL, gj_l, k1) + jb;
                entry(k0, a);
                entry(k1, b);
            } else {
                entry(k0, a);
            }
            flush_j2(d, gA, gB, two, ia, a, b);
        }
        flush_i(d, gS, ia, jb, touched, fi);  // every 32 entries (EPC)
        touched = 0;
        if (PRUNE && lane < ne) d.ent_hdr[ebase + eb + lane].y = (hy_l & ~0xff00) | (int)(keep_l << 8);
    }
}

// the re-pruning form, out of line: the common form's code stays as it is
template <int WARPS>
__device__ __noinline__ void item_entries_prune(const Dev &d, PairShared<WARPS> &sh, const SysDev &S, int4 it,
                                                int gS) {
    float elj = 0.f, erf = 0.f;
    int npair = 0;
    item_entries<false, WARPS, 8, true>(d, sh, S, it, gS, elj, erf, npair);
}

// work items of the normal pairs, handed out by a global counter
template <bool ENERGY, int WARPS, int MSHIFT>
__device__ __forceinline__ void normal_items(const Dev &d, int w0, int w1, int nblk, PairShared<WARPS> &sh) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw = w1 - w0;
    const int total = sh.pre[nw];
    // the next item's index is fetched one item ahead, so that the atomic's
    // round trip overlaps the current item's work
    int v_next = 0;
    if (lane == 0) v_next = (int)atomicAdd(&d.counters[CTR_ITEM], 1ull);
    for (;;) {
        const int v = __shfl_sync(FULL, v_next, 0);
        if (v >= total) break;
        if (lane == 0) v_next = (int)atomicAdd(&d.counters[CTR_ITEM], 1ull);
        int lo = 0, hi = nw - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (sh.pre[mid] <= v) lo = mid; else hi = mid - 1;
        }
        const int w = w0 + lo;
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        const int4 it = d.items[W.item_base + (v - sh.pre[lo])];
        if (!la_in(d, it.x - W.sc_off, W.sc_cap) || !la_in(d, it.z - 1, d.ent_cap) || !la_in(d, it.y, it.z))
            continue;  // item skipped
        const int sc = it.x;
        const int gS = W.slot_off + (sc - W.sc_off) * SC;
        __syncwarp();
        sh.sxq[wib][lane] = d.xq[gS + lane];
        sh.sxq[wib][lane + 32] = d.xq[gS + lane + 32];
        sh.slj[wib][lane] = d.lj[gS + lane];
        sh.slj[wib][lane + 32] = d.lj[gS + lane + 32];
        float elj = 0.f, erf = 0.f;
        int npair = 0;
        if (MSHIFT == 8 && d.prune_now[w] != 0ull) item_entries_prune<WARPS>(d, sh, S, it, gS);
        else item_entries<ENERGY, WARPS, MSHIFT, false>(d, sh, S, it, gS, elj, erf, npair);
        if (ENERGY) {
            const double el = warp_sum((double)elj), er = warp_sum((double)erf);
            int np = npair;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(FULL, np, o);
            if (lane == 0) {
                atomicAdd((unsigned long long *)&d.eterm[N_ETERMS * w + 0],
                          (unsigned long long)__double2ll_rn(el * E_TO_FIX));
                atomicAdd((unsigned long long *)&d.eterm[N_ETERMS * w + 1],
                          (unsigned long long)__double2ll_rn(er * E_TO_FIX));
                atomicAdd(&d.counters[1], (unsigned long long)np);
            }
        }
    }
    // the last warp out resets the work counters for the next launch
    if (lane == 0) {
        __threadfence();
        const unsigned long long done = atomicAdd(&d.counters[CTR_DONE], 1ull);
        if (done == (unsigned long long)nblk * WARPS - 1ull) {
            d.counters[CTR_ITEM] = 0ull;
            d.counters[CTR_DONE] = 0ull;
            __threadfence();
        }
    }
}

// Fused launch: a walker's terms (walker_work) need all its alchemical
// items, and a stage's lambda update (lambda_work) needs all its walkers.
// Each finished item, plus one extra trigger item per walker, arrives on
// the walker's counter; the warp that arrives last does the walker's work and
// arrives on the stage's counter, whose last arrival does the stage's work.
// Writers fence before arriving; counters are reset by the last arrival.
// No warp waits for another.
__device__ __forceinline__ void arrive_walker(const Dev &d, int w, int lane) {
    __threadfence();
    unsigned old = 0;
    if (lane == 0) old = atomicAdd(&d.wdone[w], 1u);
    old = __shfl_sync(FULL, old, 0);
    const WalkerDev &W = d.walk[w];
    if (old != (unsigned)d.sys[W.sys].n_alch) return;  // n_alch + 1 arrivals
    if (lane == 0) d.wdone[w] = 0u;
    __threadfence();
    walker_work<false>(d, w, lane);
    __threadfence();
    const int si = W.stage;
    const StageDev &st = d.stage[si];
    unsigned old2 = 0;
    if (lane == 0) old2 = atomicAdd(&d.sdone[si], 1u);
    old2 = __shfl_sync(FULL, old2, 0);
    if (old2 != (unsigned)(st.w1 - st.w0 - 1)) return;
    if (lane == 0) d.sdone[si] = 0u;
    __threadfence();
    lambda_work<true>(d, si, 0, lane, 32);
}

template <bool ENERGY, int WARPS, bool FUSED>
__device__ __forceinline__ void alch_items(const Dev &d, int w0, int w1, int a0, int a1, int blk, int nblk) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = nblk * WARPS;
    const int aend = FUSED ? a1 + (w1 - w0) : a1;
    for (int it = a0 + blk * WARPS + wib; it < aend; it += nwarps) {
        if (FUSED && it >= a1) {  // trigger item of walker w0 + (it - a1)
            arrive_walker(d, w0 + (it - a1), lane);
            continue;
        }
        int lo = w0, hi = w1 - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (d.walk[mid].alch_base <= it) lo = mid; else hi = mid - 1;
        }
        const int w = lo;
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        const int r = it - W.alch_base;
        int a = d.alch_atoms[S.alch_off + r];
        bool item_ok = la_in(d, a, S.n_atoms);
        if (!item_ok) a = 0;
        int ga = d.slot_of_atom[W.atom_base + a];
        if (!la_in(d, ga, d.n_slots)) ga = W.slot_off, item_ok = false;  // no pairs, still arrives
        const float4 xa = d.xq[ga];
        const float2 la = d.lj[ga];
        double lvd, led, dlvd, dled;
        lambda_path(d.lam[w], S.b_v, S.b_e, lvd, led, dlvd, dled);
        const float le = (float)led;
        // integer soft-core powers by repeated multiplication: the FP64 pipe
        // is narrow on this GPU, and the warps of a block share one SM's
        const float lvn = (float)ipow(lvd, S.sc_n);
        const float dlvn = (float)((double)S.sc_n * ipow(lvd, S.sc_n - 1));
        const float sa = (float)((double)S.sc_alpha * ipow(1.0 - lvd, S.sc_m));
        const float dsdl = (float)(-(double)S.sc_m * S.sc_alpha * ipow(1.0 - lvd, S.sc_m - 1));
        const float eps_a = 0.25f * la.y * la.y;
        const double inv2eps = 0.5 / (double)eps_a;  // d e4 / d eps_a = e4 / (2 eps_a)
        const float rc2 = S.rc2, krf = S.krf, crf = S.crf;
        float fax = 0.f, fay = 0.f, faz = 0.f;
        double sv = 0.0, se = 0.0, usc_s = 0.0, urf_s = 0.0;
        double th0 = 0.0, th1 = 0.0, th2 = 0.0, th3 = 0.0, th4 = 0.0, th5 = 0.0;
        int npair = 0;
        const int cnt = item_ok ? d.alch_cnt[it] : 0;
        const int *lst = d.alch_slot + (size_t)it * d.alch_cap;
        for (int k = lane; k < cnt; k += 32) {
            const int gb = lst[k];
            if (!la_in(d, gb, d.n_slots)) continue;
            const float4 xb = d.xq[gb];
            const float2 lb = d.lj[gb];
            const float dx = min_image(xa.x - xb.x, S.boxf, S.box_invf);
            const float dy = min_image(xa.y - xb.y, S.boxf, S.box_invf);
            const float dz = min_image(xa.z - xb.z, S.boxf, S.box_invf);
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= rc2) continue;
            ++npair;
            const float rinv = rsqrtf(r2);
            const float r2inv = rinv * rinv;
            const float rf_shape = rinv + krf * r2 - crf;
            const float qq = xa.w * xb.w;
            const float rf_u = qq * rf_shape;
            const float rf_f = qq * (rinv * r2inv - 2.0f * krf);
            const float sg = la.x + lb.x;
            const float e4 = la.y * lb.y;
            float sc_f = 0.f, usc = 0.f, dsc = 0.f, g = 0.f, g1 = 0.f, g2 = 0.f, rho6 = 0.f;
            if (e4 > 0.f) {
                const float q2 = r2 / (sg * sg);
                rho6 = q2 * q2 * q2;
                const float s = sa + rho6;
                const float is = 1.0f / s;
                g = is * is - is;
                g1 = is * is - 2.0f * is * is * is;
                g2 = 6.0f * is * is * is * is - 2.0f * is * is * is;
                usc = lvn * e4 * g;
                sc_f = -lvn * e4 * g1 * 6.0f * rho6 * r2inv;
                dsc = dlvn * e4 * g + lvn * e4 * g1 * dsdl;
            }
            const float fs = sc_f + le * rf_f;
            fax = fmaf(fs, dx, fax);
            fay = fmaf(fs, dy, fay);
            faz = fmaf(fs, dz, faz);
            add_force(d, gb, -fs * dx, -fs * dy, -fs * dz);
            sv += (double)dsc;
            se += (double)rf_u;
            usc_s += (double)usc;
            urf_s += (double)(le * rf_u);
            if (S.theta_stats || ENERGY) {
                if (e4 > 0.f) {
                    th0 += (double)usc * inv2eps;
                    th3 += (double)dsc * inv2eps;
                    const float ds_dsig = -6.0f * rho6 / sg;
                    th1 += 0.5 * (double)(lvn * e4 * g1 * ds_dsig);
                    th4 += 0.5 * (double)(dlvn * e4 * g1 * ds_dsig + lvn * e4 * g2 * ds_dsig * dsdl);
                }
                // d/dq_a of coul q_a q_b shape = sqrt(coul) * (q_b sqrt(coul)) * shape
                const float qb_c = S.sqrt_coul * xb.w;
                th2 += (double)(le * qb_c * rf_shape);
                th5 += (double)(qb_c * rf_shape);
            }
        }
        fax = warp_sumf(fax);
        fay = warp_sumf(fay);
        faz = warp_sumf(faz);
        sv = warp_sum(sv);
        se = warp_sum(se);
        usc_s = warp_sum(usc_s);
        urf_s = warp_sum(urf_s);
        if (S.theta_stats || ENERGY) {
            th0 = warp_sum(th0); th1 = warp_sum(th1); th2 = warp_sum(th2);
            th3 = warp_sum(th3); th4 = warp_sum(th4); th5 = warp_sum(th5);
        }
        if (ENERGY) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) npair += __shfl_xor_sync(FULL, npair, o);
        }
        if (lane == 0) {
            add_force(d, ga, fax, fay, faz);
            double *o = d.alch_out + 4 * (size_t)it;
            o[0] = sv;
            o[1] = se;
            o[2] = usc_s;
            o[3] = urf_s;
            if (S.theta_stats || ENERGY) {
                double *t = d.alch_th + 6 * (size_t)it;
                t[0] = th0; t[1] = th1; t[2] = th2; t[3] = th3; t[4] = th4; t[5] = th5;
            }
            if (ENERGY) atomicAdd(&d.counters[2], (unsigned long long)npair);
        }
        if (FUSED) arrive_walker(d, w, lane);
    }
}

// bonded terms in the fused launch: blocks [0, nblk) of the bonded range
__device__ __forceinline__ void bonded_items(const Dev &d, int w0, int w1, int blk, int nblk) {
    const int b0 = d.walk[w0].bo_off;
    const int b1 = d.walk[w1 - 1].bo_off + d.walk[w1 - 1].n_bo;
    const int nthr = nblk * blockDim.x;
    for (int t = b0 + blk * blockDim.x + threadIdx.x; t < b1; t += nthr) bonded_term<false>(d, t, w0, w1);
}

// WARPS x 32 threads per CTA; MINB: resident CTAs per SM the register
// allocation is sized for.  Variants (autotuned): 8 warps / 3 CTAs (80
// registers), 4 warps / 7 CTAs (72), 4 warps / 8 CTAs (64).
template <bool ENERGY, int WARPS, int MINB, bool FUSED>
__global__ void __launch_bounds__(WARPS * 32, MINB) k_pairs(Dev d, int w0, int w1, int nblk_pairs, int a0, int a1,
                                                          int nblk_bonded) {
    __shared__ PairShared<WARPS> sh;
    // grid: [alchemical items][bonded terms][normal pairs]; the first two
    // come first so that they run alongside the normal pairs
    const int nblk_alch = gridDim.x - nblk_pairs - nblk_bonded;
    if ((int)blockIdx.x < nblk_alch) {
        alch_items<ENERGY, WARPS, FUSED>(d, w0, w1, a0, a1, blockIdx.x, nblk_alch);
        return;
    }
    if (FUSED && (int)blockIdx.x < nblk_alch + nblk_bonded) {
        bonded_items(d, w0, w1, blockIdx.x - nblk_alch, nblk_bonded);
        return;
    }
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = w0; w < w1; ++w) {
            sh.pre[w - w0] = acc;
            acc += d.n_items[w];
        }
        sh.pre[w1 - w0] = acc;
    }
    __syncthreads();
    normal_items<ENERGY, WARPS, FUSED ? 8 : 16>(d, w0, w1, nblk_pairs, sh);
}

template <bool ENERGY, int WARPS, int MINB>
static void launch_pairs_v(const Dev &d, const HostView &hv, int w0, int w1, cudaStream_t s, bool fused = false) {
    int nblk = hv.pair_blocks * 8 / WARPS;  // pair_blocks counts 8-warp CTAs
    if (w1 - w0 < hv.n_walkers) {           // a subset of walkers: size the grid to its work
        int items = 0;
        for (int w = w0; w < w1; ++w) items += hv.item_cap[w];
        int need = (items + WARPS - 1) / WARPS;
        nblk = need < nblk ? need : nblk;
        nblk = nblk < 1 ? 1 : nblk;
    }
    const int a0 = hv.alch_base[w0], a1 = hv.alch_base[w1 - 1] + hv.n_alch[w1 - 1];
    const int ablk = (a1 - a0 + (fused ? w1 - w0 : 0) + WARPS - 1) / WARPS;
    int bblk = 0;
    if (fused) {  // bonded terms: about four per thread
        const int nbo = hv.bo_off[w1 - 1] + hv.n_bo[w1 - 1] - hv.bo_off[w0];
        bblk = (nbo + 4 * WARPS * 32 - 1) / (4 * WARPS * 32);
        bblk = bblk > hv.n_sm ? hv.n_sm : bblk;
    }
    const int grid = ablk + bblk + nblk;
    if (fused) k_pairs<ENERGY, WARPS, MINB, true><<<grid, WARPS * 32, 0, s>>>(d, w0, w1, nblk, a0, a1, bblk);
    else k_pairs<ENERGY, WARPS, MINB, false><<<grid, WARPS * 32, 0, s>>>(d, w0, w1, nblk, a0, a1, 0);
}

void launch_pairs_fused(const Dev &d, const HostView &hv, int n_stages, cudaStream_t s) {
    const int W = hv.n_walkers;
    (void)n_stages;
    if (hv.pair_variant == 1) launch_pairs_v<false, 4, 7>(d, hv, 0, W, s, true);
    else if (hv.pair_variant == 2) launch_pairs_v<false, 4, 8>(d, hv, 0, W, s, true);
    else launch_pairs_v<false, 8, 3>(d, hv, 0, W, s, true);
}

void launch_pairs(const Dev &d, const HostView &hv, int w0, int w1, bool energy, cudaStream_t s) {
    if (energy) launch_pairs_v<true, 8, 3>(d, hv, w0, w1, s);
    else if (hv.pair_variant == 1) launch_pairs_v<false, 4, 7>(d, hv, w0, w1, s);
    else if (hv.pair_variant == 2) launch_pairs_v<false, 4, 8>(d, hv, w0, w1, s);
    else launch_pairs_v<false, 8, 3>(d, hv, w0, w1, s);
}

}  // namespace labf
