// labf_dyn.cuh -- per-term, per-walker and per-stage device work shared by
// the separate kernels (k_dyn.cu) and the fused pair launch (k_pairs.cu).
#pragma once
#include "labf_internal.cuh"

namespace labf {

// ---------------------------------------------------------------------------
// bonds (1/2 k (r - r0)^2), angles (1/2 k (theta - theta0)^2) and positional
// restraints (1/2 k |x - x0|^2): term t of the bonded items of walkers
// [w0, w1)
// ---------------------------------------------------------------------------
template <bool ENERGY>
__device__ __forceinline__ void bonded_term(const Dev &d, int t, int w0, int w1) {
    int lo = w0, hi = w1 - 1;  // walker owning item t
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d.walk[mid].bo_off <= t) lo = mid; else hi = mid - 1;
    }
    const int w = lo;
    const WalkerDev &W = d.walk[w];
    const SysDev &S = d.sys[W.sys];
    const int *soa = d.slot_of_atom + W.atom_base;
    int k = t - W.bo_off;
    float e = 0.f;
    int eterm = 4;
    if (k < S.n_bonds) {
        const int2 ij = d.bond_ij[S.bond_off + k];
        const float2 p = d.bond_p[S.bond_off + k];
        const int gi = checked_slot(d, soa[ij.x]), gj = checked_slot(d, soa[ij.y]);
        const float4 xi = d.xq[gi], xj = d.xq[gj];
        float dx = min_image(xi.x - xj.x, S.boxf, S.box_invf);
        float dy = min_image(xi.y - xj.y, S.boxf, S.box_invf);
        float dz = min_image(xi.z - xj.z, S.boxf, S.box_invf);
        float r = sqrtf(dx * dx + dy * dy + dz * dz);
        float dr = r - p.x;
        float fs = -p.y * dr / r;
        add_force(d, gi, fs * dx, fs * dy, fs * dz);
        add_force(d, gj, -fs * dx, -fs * dy, -fs * dz);
        if (ENERGY) e = 0.5f * p.y * dr * dr;
    } else if ((k -= S.n_bonds) < S.n_angles) {
        const int4 ijk = d.angle_ijk[S.angle_off + k];
        const float2 p = d.angle_p[S.angle_off + k];
        const int gi = checked_slot(d, soa[ijk.x]), gj = checked_slot(d, soa[ijk.y]), gk = checked_slot(d, soa[ijk.z]);
        const float4 xi = d.xq[gi], xj = d.xq[gj], xk = d.xq[gk];
        float ux = min_image(xi.x - xj.x, S.boxf, S.box_invf);
        float uy = min_image(xi.y - xj.y, S.boxf, S.box_invf);
        float uz = min_image(xi.z - xj.z, S.boxf, S.box_invf);
        float vx = min_image(xk.x - xj.x, S.boxf, S.box_invf);
        float vy = min_image(xk.y - xj.y, S.boxf, S.box_invf);
        float vz = min_image(xk.z - xj.z, S.boxf, S.box_invf);
        float nu2 = ux * ux + uy * uy + uz * uz, nv2 = vx * vx + vy * vy + vz * vz;
        float inu = rsqrtf(nu2), inv = rsqrtf(nv2);
        float cs = (ux * vx + uy * vy + uz * vz) * inu * inv;
        cs = fminf(1.f, fmaxf(-1.f, cs));
        float th = acosf(cs);
        float dth = th - p.x;
        float sn = sqrtf(fmaxf(1.f - cs * cs, 1e-12f));
        float g = p.y * dth / sn;  // dU/dtheta / sin(theta)
        float a11 = g * inu * inv, a12 = g * cs * inu * inu, a22 = g * cs * inv * inv;
        float fix = a11 * vx - a12 * ux, fiy = a11 * vy - a12 * uy, fiz = a11 * vz - a12 * uz;
        float fkx = a11 * ux - a22 * vx, fky = a11 * uy - a22 * vy, fkz = a11 * uz - a22 * vz;
        add_force(d, gi, fix, fiy, fiz);
        add_force(d, gk, fkx, fky, fkz);
        add_force(d, gj, -fix - fkx, -fiy - fky, -fiz - fkz);
        if (ENERGY) {
            e = 0.5f * p.y * dth * dth;
            eterm = 5;
        }
    } else {
        k -= S.n_angles;
        const int ai = d.posres_idx[S.posres_off + k];
        const float4 x0 = d.posres_x0[S.posres_off + k];
        const int gi = checked_slot(d, soa[ai]);
        const float4 xi = d.xq[gi];
        float dx = min_image(xi.x - x0.x, S.boxf, S.box_invf);
        float dy = min_image(xi.y - x0.y, S.boxf, S.box_invf);
        float dz = min_image(xi.z - x0.z, S.boxf, S.box_invf);
        add_force(d, gi, -S.posres_k * dx, -S.posres_k * dy, -S.posres_k * dz);
        if (ENERGY) {
            e = 0.5f * S.posres_k * (dx * dx + dy * dy + dz * dz);
            eterm = 6;
        }
    }
    if (ENERGY) atomicAdd((unsigned long long *)&d.eterm[N_ETERMS * w + eterm],
                          (unsigned long long)__double2ll_rn((double)e * E_TO_FIX));
}

// ---------------------------------------------------------------------------
// per walker, one warp: flat-bottom COM restraint, lambda-dependent distance
// restraint, lambda-switched well, and the sum of the alchemical partials
// into s = dU/dlambda.  Lane-strided loops and fixed shuffle trees: the
// result is deterministic.  The alchemical partials may come from other SMs
// of the same launch: they are read past L1.
// ---------------------------------------------------------------------------
template <bool ENERGY>
__device__ __forceinline__ void walker_work(const Dev &d, int w, int lane) {
    const WalkerDev &W = d.walk[w];
    const SysDev &S = d.sys[W.sys];
    const int *soa = d.slot_of_atom + W.atom_base;
    double lv, le, dlv, dle;
    lambda_path(d.lam[w], S.b_v, S.b_e, lv, le, dlv, dle);
    double e_rest = 0.0;

    // ---- flat-bottom restraint on |COM_a - COM_b| ----
    if (S.n_fb_a > 0 && S.n_fb_b > 0) {
        double com[2][4];
        for (int grp = 0; grp < 2; ++grp) {
            const int off = S.fb_off + (grp ? S.n_fb_a : 0);
            const int ng = grp ? S.n_fb_b : S.n_fb_a;
            const float4 r0 = d.xq[checked_slot(d, soa[d.fb_idx[off]])];
            double acc[4] = {0, 0, 0, 0};
            for (int k = lane; k < ng; k += 32) {
                const int a = d.fb_idx[off + k];
                const float4 xa = d.xq[checked_slot(d, soa[a])];
                const double m = 1.0 / (double)d.ap[S.atom_off + a].w;
                acc[0] += m * min_image(xa.x - r0.x, S.boxf, S.box_invf);
                acc[1] += m * min_image(xa.y - r0.y, S.boxf, S.box_invf);
                acc[2] += m * min_image(xa.z - r0.z, S.boxf, S.box_invf);
                acc[3] += m;
            }
            for (int c = 0; c < 4; ++c) com[grp][c] = warp_sum(acc[c]);
            com[grp][0] = r0.x + com[grp][0] / com[grp][3];
            com[grp][1] = r0.y + com[grp][1] / com[grp][3];
            com[grp][2] = r0.z + com[grp][2] / com[grp][3];
        }
        double dv[3];
        for (int c = 0; c < 3; ++c) {
            const double t = com[0][c] - com[1][c];
            dv[c] = t - S.box * nearbyint(t * S.box_inv);
        }
        const double dd = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        if (dd > S.fb_d0) {
            const double ex = dd - S.fb_d0;
            const double fmag = S.fb_k * ex / dd;
            for (int grp = 0; grp < 2; ++grp) {
                const int off = S.fb_off + (grp ? S.n_fb_a : 0);
                const int ng = grp ? S.n_fb_b : S.n_fb_a;
                const double sgn = grp ? 1.0 : -1.0;
                const double mt = com[grp][3];
                for (int k = lane; k < ng; k += 32) {
                    const int a = d.fb_idx[off + k];
                    const double wgt = (1.0 / (double)d.ap[S.atom_off + a].w) / mt;
                    add_force(d, checked_slot(d, soa[a]), (float)(sgn * fmag * dv[0] * wgt), (float)(sgn * fmag * dv[1] * wgt),
                              (float)(sgn * fmag * dv[2] * wgt));
                }
            }
            e_rest = 0.5 * S.fb_k * ex * ex;
        }
    }

    double dl_dir = 0.0, e_lh = 0.0, dk1 = 0.0, d2k1 = 0.0;
    // ---- lambda-dependent distance restraint (Sec. 4.2): pairs kept at
    // least d_min = delta/2 (1 - cos 2 pi lambda) apart ----
    if (S.n_lr > 0) {
        const double lam = d.lam[w];
        const double dmin = 0.5 * S.lr_delta * (1.0 - cospi(2.0 * lam));
        const double ddmin = S.lr_delta * 3.14159265358979323846 * sinpi(2.0 * lam);
        for (int k = lane; k < S.n_lr; k += 32) {
            const int2 ab = d.lr_ij[S.lr_off + k];
            const int ga = checked_slot(d, soa[ab.x]), gb = checked_slot(d, soa[ab.y]);
            const float4 xa = d.xq[ga], xb = d.xq[gb];
            const float dx = min_image(xa.x - xb.x, S.boxf, S.box_invf);
            const float dy = min_image(xa.y - xb.y, S.boxf, S.box_invf);
            const float dz = min_image(xa.z - xb.z, S.boxf, S.box_invf);
            const double r = sqrt((double)dx * dx + (double)dy * dy + (double)dz * dz);
            if (r < dmin) {
                const double ex = r - dmin;
                e_lh += 0.5 * S.lr_k * ex * ex;
                dl_dir += -S.lr_k * ex * ddmin;
                const float fs = (float)(-S.lr_k * ex / r);
                add_force(d, ga, fs * dx, fs * dy, fs * dz);
                add_force(d, gb, -fs * dx, -fs * dy, -fs * dz);
            }
        }
    }
    // ---- lambda-switched harmonic well (uses lambda itself) ----
    if (S.n_lh > 0) {
        const double lam = d.lam[w];
        const double kl = (1.0 - lam) * S.lh_k0 + lam * S.lh_k1;
        for (int k = lane; k < S.n_lh; k += 32) {
            const int a = d.lh_idx[S.lh_off + k];
            const int g = checked_slot(d, soa[a]);
            const float4 xa = d.xq[g], x0 = d.lh_x0[S.lh_off + k];
            float dx = min_image(xa.x - x0.x, S.boxf, S.box_invf);
            float dy = min_image(xa.y - x0.y, S.boxf, S.box_invf);
            float dz = min_image(xa.z - x0.z, S.boxf, S.box_invf);
            if (S.lh_dims < 3) dz = 0.f;
            if (S.lh_dims < 2) dy = 0.f;
            const double r2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
            add_force(d, g, (float)(-kl * dx), (float)(-kl * dy), (float)(-kl * dz));
            dl_dir += 0.5 * (S.lh_k1 - S.lh_k0) * r2;
            e_lh += 0.5 * kl * r2;
            dk1 += 0.5 * lam * r2;
            d2k1 += 0.5 * r2;
        }
    }
    const double v0 = warp_sum(dl_dir), v1 = warp_sum(e_lh) + e_rest, v2 = warp_sum(dk1), v3 = warp_sum(d2k1);
    if (lane == 0) {
        // ---- s = dU/dlambda: alchemical partials in atom order ----
        double sv = 0.0, se = 0.0, usc = 0.0, urf = 0.0;
        for (int r = 0; r < S.n_alch; ++r) {
            const double *o = d.alch_out + 4 * (size_t)(W.alch_base + r);
            sv += __ldcg(o + 0);
            se += __ldcg(o + 1);
            usc += __ldcg(o + 2);
            urf += __ldcg(o + 3);
        }
        d.s[w] = dlv * sv + dle * se + v0;
        if (S.theta_stats || ENERGY) {
            double *th = d.wth + (size_t)w * 2 * d.P_max;
            for (int r = 0; r < S.n_alch; ++r) {
                const double *o = d.alch_th + 6 * (size_t)(W.alch_base + r);
                th[3 * r + 0] = __ldcg(o + 0);
                th[3 * r + 1] = __ldcg(o + 1);
                th[3 * r + 2] = __ldcg(o + 2);
                th[d.P_max + 3 * r + 0] = dlv * __ldcg(o + 3);
                th[d.P_max + 3 * r + 1] = dlv * __ldcg(o + 4);
                th[d.P_max + 3 * r + 2] = dle * __ldcg(o + 5);
            }
            th[S.P - 1] = v2;
            th[d.P_max + S.P - 1] = v3;
        }
        if (ENERGY) {
            long long *et = d.eterm + N_ETERMS * w;
            atomicAdd((unsigned long long *)&et[2], (unsigned long long)__double2ll_rn(usc * E_TO_FIX));
            atomicAdd((unsigned long long *)&et[3], (unsigned long long)__double2ll_rn(urf * E_TO_FIX));
            atomicAdd((unsigned long long *)&et[6], (unsigned long long)__double2ll_rn(v1 * E_TO_FIX));
            d.dl_direct[w] = v0;
        }
    }
}

// ---------------------------------------------------------------------------
// ABF: fold the samples of a stage's walkers, merge every shared_freq steps,
// bias = min(1, n/n_full) * mean, final B of lambda.
// prime = 1: only G = -s + bias (no sample, no step).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double abf_bias(const Dev &d, const SysDev &S, const StageDev &st, int w) {
    if (!S.abf_on) return 0.0;
    const int k = bin_of(d.lam[w], st);
    const size_t lk = (size_t)w * d.max_bins + k;
    const double sum = d.abf_sum[st.bin_off + k] + d.dl_sum[lk];
    const double cnt = (double)(d.abf_count[st.bin_off + k] + d.dl_count[lk]);
    if (cnt <= 0.0) return 0.0;
    return fmin(1.0, cnt / S.n_full) * sum / cnt;
}

template <bool WARP>
__device__ __forceinline__ void group_sync() {
    if (WARP) __syncwarp(); else __syncthreads();
}

// the work of stage si by a group of nt threads (a warp or a block); every
// bin, parameter and walker is handled whole by one thread, so the result
// does not depend on nt.  s and the theta samples may come from other SMs
// of the same launch: they are read past L1.
template <bool WARP>
__device__ __forceinline__ void lambda_work(const Dev &d, int si, int prime, int tid, int nt) {
    const StageDev &st = d.stage[si];
    if (st.w1 <= st.w0) return;  // (create refuses stages without walkers)
    const SysDev &S = d.sys[st.sys];
    if (!prime) {
        // fold each walker's sample into its own statistics (independent)
        for (int w = st.w0 + tid; w < st.w1; w += nt) {
            const int k = bin_of(d.lam[w], st);
            const size_t lk = (size_t)w * d.max_bins + k;
            const double sv = __ldcg(d.s + w);
            d.dl_sum[lk] += sv;
            d.dl_sumsq[lk] += sv * sv;
            d.dl_count[lk] += 1ull;
        }
        // theta statistics: per parameter, walkers in order
        if (S.theta_stats) {
            for (int p = tid; p < S.P; p += nt) {
                for (int w = st.w0; w < st.w1; ++w) {
                    const size_t b = (size_t)(st.bin_off + bin_of(d.lam[w], st)) * d.P_max + p;
                    const double *th = d.wth + (size_t)w * 2 * d.P_max;
                    const double thp = __ldcg(th + p);
                    d.th_d2[b] += __ldcg(th + d.P_max + p);
                    d.th_d[b] += thp;
                    d.th_sd[b] += __ldcg(d.s + w) * thp;
                }
            }
        }
        group_sync<WARP>();
        const unsigned long long stepn = d.step[st.w0] + 1ull;
        const int K = S.shared_freq;  // 0: merged only by the host (la_abf_import)
        if (K > 0 && stepn % (unsigned long long)K == 0ull) {
            for (int k = tid; k < st.n_bins; k += nt) {
                double s1 = d.abf_sum[st.bin_off + k], s2 = d.abf_sumsq[st.bin_off + k];
                unsigned long long c = d.abf_count[st.bin_off + k];
                for (int w = st.w0; w < st.w1; ++w) {
                    const size_t lk = (size_t)w * d.max_bins + k;
                    s1 += d.dl_sum[lk];
                    s2 += d.dl_sumsq[lk];
                    c += d.dl_count[lk];
                    d.dl_sum[lk] = 0.0;
                    d.dl_sumsq[lk] = 0.0;
                    d.dl_count[lk] = 0ull;
                }
                d.abf_sum[st.bin_off + k] = s1;
                d.abf_sumsq[st.bin_off + k] = s2;
                d.abf_count[st.bin_off + k] = c;
            }
        }
        group_sync<WARP>();
    }
    for (int w = st.w0 + tid; w < st.w1; w += nt) {
        const double G = -__ldcg(d.s + w) + abf_bias(d, S, st, w);
        d.G[w] = G;
        if (!prime) {
            if (S.lambda_dynamics) d.plam[w] += 0.5 * S.dt_d * G;
            d.step[w] += 1ull;
            d.pending[w] = 1;
        }
    }
}

}  // namespace labf
