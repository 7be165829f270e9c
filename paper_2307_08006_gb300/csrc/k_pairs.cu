// k_pairs.cu -- the pair pass: LJ + reaction-field forces of normal pairs
// over the cluster-pair list, and, in the same launch, the alchemically
// scaled pairs with the walker's dU/dlambda partials (Sec. 3.1.2, Eq.
// lambda-abf: the engine provides dV/dlambda every step).
//
// Normal pairs: one warp per work item (a chunk of one super-cluster's
// j-list).  The super-cluster's 64 slots sit in shared memory; lane
// (ia, jb) = (lane & 7, lane >> 3) owns i-atom ia of each i-cluster and
// j-atom jb of the current j-cluster.  For each entry the warp loops over
// the i-clusters flagged in the entry, so one j-cluster load and one j-force
// reduction serve up to 8 x 32 pairs; the eight i-force accumulators stay in
// registers for the whole item.  Forces are accumulated in FP32 and added to
// the 64-bit fixed-point force array with integer atomics (order-free, so
// results are bit-reproducible).
//
// Per in-cutoff pair (force only), 38 FP32 flops (FMA = 2) plus one rsqrt:
//   d = x_i - x_j (3), r2 (5), 1/r2 (1), sigma_ij = s_i + s_j, its square,
//   (sigma/r)^2, ^6 (5), 4 eps_ij (1), 4eps (sigma/r)^6 (12 (sigma/r)^6 - 6)/r2
//   (5), q_i q_j (1/r^3 - 2 k_rf) (4), sum (1), f_i += f d, f_j -= f d (12).
//
// Alchemical pairs: one warp per (walker, alchemical atom); lanes stride over
// its environment list.  Soft-core LJ lambda_v^n 4 eps (s^-2 - s^-1) with
// s = alpha (1 - lambda_v)^m + (r/sigma)^6, RF scaled by lambda_e; per-lane
// FP64 sums of dU/dlambda_v, dU/dlambda_e, energies and theta derivatives,
// reduced with a fixed shuffle tree (deterministic).
#include "labf_internal.cuh"
#include "labf_launch.h"

namespace labf {

constexpr int PAIR_WARPS = 8;

template <int IC_>
__device__ __forceinline__ unsigned pick_mask(const uint4 &m0, const uint4 &m1) {
    return IC_ == 0 ? m0.x : IC_ == 1 ? m0.y : IC_ == 2 ? m0.z : IC_ == 3 ? m0.w
         : IC_ == 4 ? m1.x : IC_ == 5 ? m1.y : IC_ == 6 ? m1.z : m1.w;
}

template <bool ENERGY>
__device__ __forceinline__ void normal_items(const Dev &d, int w0, int w1, int nblk, float4 (*sxq)[SC],
                                             float2 (*slj)[SC], const int *pre) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int ia = lane & 7, jb = lane >> 3;
    const int nw = w1 - w0;
    const int total = pre[nw];
    const int nwarps = nblk * PAIR_WARPS;
    for (int v = blockIdx.x * PAIR_WARPS + wib; v < total; v += nwarps) {
        int lo = 0, hi = nw - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= v) lo = mid; else hi = mid - 1;
        }
        const int w = w0 + lo;
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        const int4 it = d.items[W.item_base + (v - pre[lo])];
        const int sc = it.x;
        const int gS = W.slot_off + (sc - W.sc_off) * SC;
        __syncwarp();
        sxq[wib][lane] = d.xq[gS + lane];
        sxq[wib][lane + 32] = d.xq[gS + lane + 32];
        slj[wib][lane] = d.lj[gS + lane];
        slj[wib][lane + 32] = d.lj[gS + lane + 32];
        __syncwarp();
        const float L = S.boxf, rc2 = S.rc2, krf2 = 2.0f * S.krf, krf = S.krf, crf = S.crf;
        float fi[NIC][3];
#pragma unroll
        for (int ic = 0; ic < NIC; ++ic) fi[ic][0] = fi[ic][1] = fi[ic][2] = 0.f;
        unsigned touched = 0;
        float elj = 0.f, erf = 0.f;
        int npair = 0;
        const size_t ebase = (size_t)sc * d.ent_cap;
        for (int e = it.y; e < it.z; ++e) {
            const int2 hdr = d.ent_hdr[ebase + e];
            const uint4 m0 = d.ent_mask[2 * (ebase + e)], m1 = d.ent_mask[2 * (ebase + e) + 1];
            const int gj = hdr.x + jb;
            float4 xj = d.xq[gj];
            const float2 lj_j = d.lj[gj];
            const int code = hdr.y & 255;
            const int sx = code % 3 - 1, sy = (code / 3) % 3 - 1, sz = code / 9 - 1;
            xj.x += (float)sx * L;
            xj.y += (float)sy * L;
            xj.z += (float)sz * L;
            const unsigned imask = (unsigned)hdr.y >> 8;
            touched |= imask;
            float fjx = 0.f, fjy = 0.f, fjz = 0.f;
#pragma unroll
            for (int ic = 0; ic < NIC; ++ic) {
                if (imask & (1u << ic)) {
                    unsigned m;
                    switch (ic) {
                        case 0: m = pick_mask<0>(m0, m1); break;
                        case 1: m = pick_mask<1>(m0, m1); break;
                        case 2: m = pick_mask<2>(m0, m1); break;
                        case 3: m = pick_mask<3>(m0, m1); break;
                        case 4: m = pick_mask<4>(m0, m1); break;
                        case 5: m = pick_mask<5>(m0, m1); break;
                        case 6: m = pick_mask<6>(m0, m1); break;
                        default: m = pick_mask<7>(m0, m1); break;
                    }
                    const float4 xi = sxq[wib][ic * IC + ia];
                    const float2 li = slj[wib][ic * IC + ia];
                    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const bool in = ((m >> lane) & 1u) && (r2 < rc2);
                    const float rinv = rsqrtf(r2);
                    const float r2inv = rinv * rinv;
                    const float sg = li.x + lj_j.x;
                    const float sr2 = sg * sg * r2inv;
                    const float sr6 = sr2 * sr2 * sr2;
                    const float e4 = li.y * lj_j.y;
                    const float flj = e4 * sr6 * fmaf(12.f, sr6, -6.f) * r2inv;
                    const float qq = xi.w * xj.w;
                    const float frf = qq * (rinv * r2inv - krf2);
                    float fs = flj + frf;
                    fs = in ? fs : 0.f;
                    fi[ic][0] = fmaf(fs, dx, fi[ic][0]);
                    fi[ic][1] = fmaf(fs, dy, fi[ic][1]);
                    fi[ic][2] = fmaf(fs, dz, fi[ic][2]);
                    fjx = fmaf(-fs, dx, fjx);
                    fjy = fmaf(-fs, dy, fjy);
                    fjz = fmaf(-fs, dz, fjz);
                    if (ENERGY) {
                        if (in) {
                            elj += e4 * sr6 * (sr6 - 1.f);
                            erf += qq * (rinv + krf * r2 - crf);
                            ++npair;
                        }
                    }
                }
            }
            // j-force: sum over the 8 i-lanes of each j-atom
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                fjx += __shfl_xor_sync(0xffffffffu, fjx, o);
                fjy += __shfl_xor_sync(0xffffffffu, fjy, o);
                fjz += __shfl_xor_sync(0xffffffffu, fjz, o);
            }
            if (ia < 3) {
                const float f = ia == 0 ? fjx : (ia == 1 ? fjy : fjz);
                atomicAdd(d.F + 3 * (size_t)gj + ia, (unsigned long long)__float2ll_rn(f * F_TO_FIX));
            }
        }
        // i-forces: sum over the 4 j-lanes; lane (ia, jb) writes i-clusters 2jb, 2jb+1
#pragma unroll
        for (int ic = 0; ic < NIC; ++ic) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                fi[ic][c] += __shfl_xor_sync(0xffffffffu, fi[ic][c], 8);
                fi[ic][c] += __shfl_xor_sync(0xffffffffu, fi[ic][c], 16);
            }
        }
#pragma unroll
        for (int ic = 0; ic < NIC; ++ic) {
            if ((ic >> 1) == jb && (touched & (1u << ic))) {
                const int gi = gS + ic * IC + ia;
                unsigned long long *p = d.F + 3 * (size_t)gi;
                atomicAdd(p + 0, (unsigned long long)__float2ll_rn(fi[ic][0] * F_TO_FIX));
                atomicAdd(p + 1, (unsigned long long)__float2ll_rn(fi[ic][1] * F_TO_FIX));
                atomicAdd(p + 2, (unsigned long long)__float2ll_rn(fi[ic][2] * F_TO_FIX));
            }
        }
        if (ENERGY) {
            const double el = warp_sum((double)elj), er = warp_sum((double)erf);
            int np = npair;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
            if (lane == 0) {
                atomicAdd((unsigned long long *)&d.eterm[N_ETERMS * w + 0],
                          (unsigned long long)__double2ll_rn(el * E_TO_FIX));
                atomicAdd((unsigned long long *)&d.eterm[N_ETERMS * w + 1],
                          (unsigned long long)__double2ll_rn(er * E_TO_FIX));
                atomicAdd(&d.counters[1], (unsigned long long)np);
            }
        }
    }
}

template <bool ENERGY>
__device__ __forceinline__ void alch_items(const Dev &d, int w0, int w1, int a0, int a1, int blk, int nblk) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = nblk * PAIR_WARPS;
    for (int it = a0 + blk * PAIR_WARPS + wib; it < a1; it += nwarps) {
        int lo = w0, hi = w1 - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (d.walk[mid].alch_base <= it) lo = mid; else hi = mid - 1;
        }
        const int w = lo;
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        const int r = it - W.alch_base;
        const int a = d.alch_atoms[S.alch_off + r];
        const int ga = d.slot_of_atom[W.atom_base + a];
        const float4 xa = d.xq[ga];
        const float2 la = d.lj[ga];
        double lvd, led, dlvd, dled;
        lambda_path(d.lam[w], S.b_v, S.b_e, lvd, led, dlvd, dled);
        const float le = (float)led;
        const float lvn = (float)pow(lvd, (double)S.sc_n);
        const float dlvn = (float)((double)S.sc_n * pow(lvd, (double)(S.sc_n - 1)));
        const float sa = (float)((double)S.sc_alpha * pow(1.0 - lvd, (double)S.sc_m));
        const float dsdl = (float)(-(double)S.sc_m * S.sc_alpha * pow(1.0 - lvd, (double)(S.sc_m - 1)));
        const float eps_a = 0.25f * la.y * la.y;
        const float rc2 = S.rc2, krf = S.krf, crf = S.crf;
        float fax = 0.f, fay = 0.f, faz = 0.f;
        double sv = 0.0, se = 0.0, usc_s = 0.0, urf_s = 0.0;
        double th0 = 0.0, th1 = 0.0, th2 = 0.0, th3 = 0.0, th4 = 0.0, th5 = 0.0;
        int npair = 0;
        const int cnt = d.alch_cnt[it];
        const int *lst = d.alch_slot + (size_t)it * d.alch_cap;
        for (int k = lane; k < cnt; k += 32) {
            const int gb = lst[k];
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
                    th0 += (double)usc / (2.0 * (double)eps_a);
                    th3 += (double)dsc / (2.0 * (double)eps_a);
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
            for (int o = 16; o > 0; o >>= 1) npair += __shfl_xor_sync(0xffffffffu, npair, o);
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
    }
}

template <bool ENERGY>
__global__ void __launch_bounds__(PAIR_WARPS * 32) k_pairs(Dev d, int w0, int w1, int nblk_pairs, int a0, int a1) {
    __shared__ float4 sxq[PAIR_WARPS][SC];
    __shared__ float2 slj[PAIR_WARPS][SC];
    __shared__ int pre[LA_MAX_WALKERS_PER_LAUNCH + 1];
    if (blockIdx.x >= nblk_pairs) {
        alch_items<ENERGY>(d, w0, w1, a0, a1, blockIdx.x - nblk_pairs, gridDim.x - nblk_pairs);
        return;
    }
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = w0; w < w1; ++w) {
            pre[w - w0] = acc;
            acc += d.n_items[w];
        }
        pre[w1 - w0] = acc;
    }
    __syncthreads();
    normal_items<ENERGY>(d, w0, w1, nblk_pairs, sxq, slj, pre);
}

void launch_pairs(const Dev &d, const HostView &hv, int w0, int w1, bool energy, cudaStream_t s) {
    int nblk = hv.pair_blocks;
    if (w1 - w0 < hv.n_walkers) {  // one walker: size the grid to its work
        int items = 0;
        for (int w = w0; w < w1; ++w) items += hv.item_cap[w];
        int need = (items + PAIR_WARPS - 1) / PAIR_WARPS;
        nblk = need < nblk ? need : nblk;
        nblk = nblk < 1 ? 1 : nblk;
    }
    const int a0 = hv.alch_base[w0], a1 = hv.alch_base[w1 - 1] + hv.n_alch[w1 - 1];
    int ablk = (a1 - a0 + PAIR_WARPS - 1) / PAIR_WARPS;
    if (energy) k_pairs<true><<<nblk + ablk, PAIR_WARPS * 32, 0, s>>>(d, w0, w1, nblk, a0, a1);
    else k_pairs<false><<<nblk + ablk, PAIR_WARPS * 32, 0, s>>>(d, w0, w1, nblk, a0, a1);
}

}  // namespace labf
