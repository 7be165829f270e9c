// k_dyn.cu -- BAOAB of atoms and lambda, bonded and restraint terms, the
// per-walker dU/dlambda sum, and the ABF fold / bias / TI helpers.
//
// Step order (Eq. lambda-abf; BAOAB as in SI Sec. S1), per MD step:
//   k_integrate : [finish B of the previous step] B A O A for atoms and lambda
//   (rebuild)   : neighbour lists if any atom moved more than skin/2
//   k_pairs     : forces, dU/dlambda partials           (k_pairs.cu)
//   k_bonded    : bonds, angles, positional restraints
//   k_walker    : flat-bottom COM restraint, lambda-switched well, dU/dlambda sum
//   k_lambda    : fold samples, bias, final B of lambda
// and once at the end of a call k_finish applies the atoms' final B.
#include "labf_internal.cuh"
#include "labf_launch.h"

namespace labf {

// ---------------------------------------------------------------------------
// atoms: BAOA (with the previous step's final B when pending), lambda: BAOA
// ---------------------------------------------------------------------------
__global__ void k_integrate(Dev d, int w0, int w1, int g0, int g1) {
    const int nthr = gridDim.x * blockDim.x;
    // lambda particles: handled by the first w1-w0 threads of the last block
    if (blockIdx.x == gridDim.x - 1) {
        int w = w0 + threadIdx.x;
        if (w < w1) {
            const SysDev &S = d.sys[d.walk[w].sys];
            if (S.lambda_dynamics) {
                const StageDev &st = d.stage[d.walk[w].stage];
                double lam = d.lam[w], p = d.plam[w];
                const double hdt = 0.5 * S.dt_d;
                p += hdt * d.G[w];
                lam += hdt * p / S.m_lambda;
                for (int it = 0; it < 64 && (lam < st.lo || lam > st.hi); ++it) {
                    if (lam < st.lo) lam = 2.0 * st.lo - lam; else lam = 2.0 * st.hi - lam;
                    p = -p;
                }
                p = S.c_lm * p + S.sd_lm * normal_lambda(S.seed, (uint32_t)d.walk[w].wlocal, d.step[w]);
                lam += hdt * p / S.m_lambda;
                for (int it = 0; it < 64 && (lam < st.lo || lam > st.hi); ++it) {
                    if (lam < st.lo) lam = 2.0 * st.lo - lam; else lam = 2.0 * st.hi - lam;
                    p = -p;
                }
                if (!(lam >= st.lo && lam <= st.hi)) set_status(d, LA_STATUS_NONFINITE);
                d.lam[w] = lam;
                d.plam[w] = p;
            }
        }
    }
    for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += nthr) {
        const int a = d.atom_of_slot[g];
        if (a < 0) continue;
        const int w = d.slot_walker[g];
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        unsigned long long *Fp = d.F + 3 * (size_t)g;
        float fx = fix_to_float(Fp[0]), fy = fix_to_float(Fp[1]), fz = fix_to_float(Fp[2]);
        if (fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))) > FIX_LIMIT) set_status(d, LA_STATUS_FIXED_OVERFLOW);
        const float2 im = d.im[g];
        float4 v = d.vv[g];
        float4 x = d.xq[g];
        const float hk = 0.5f * S.dt * im.x;
        if (d.pending[w]) {  // final B of the previous step
            v.x += hk * fx;
            v.y += hk * fy;
            v.z += hk * fz;
        }
        // B
        v.x += hk * fx;
        v.y += hk * fy;
        v.z += hk * fz;
        // A
        const float hdt = 0.5f * S.dt;
        x.x += hdt * v.x;
        x.y += hdt * v.y;
        x.z += hdt * v.z;
        // O
        const float4 z = normals4(S.seed, (uint32_t)W.wlocal, d.step[w], (uint32_t)a, 0u);
        const float sd = S.s_at * im.y;
        v.x = S.c_at * v.x + sd * z.x;
        v.y = S.c_at * v.y + sd * z.y;
        v.z = S.c_at * v.z + sd * z.z;
        // A.  Positions are not wrapped here: the cluster-pair list stores
        // periodic shifts valid for the positions it was built from, so atoms
        // are put back into [0, L) only at the next rebuild (after moving at
        // most skin/2).
        x.x += hdt * v.x;
        x.y += hdt * v.y;
        x.z += hdt * v.z;
        if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z))) set_status(d, LA_STATUS_NONFINITE);
        d.xq[g] = x;
        d.vv[g] = v;
        Fp[0] = 0ull;
        Fp[1] = 0ull;
        Fp[2] = 0ull;
        // Verlet-buffer criterion: rebuild when an atom moved more than skin/2
        const float4 r = d.xref[g];
        float dx = min_image(x.x - r.x, S.boxf, S.box_invf);
        float dy = min_image(x.y - r.y, S.boxf, S.box_invf);
        float dz = min_image(x.z - r.z, S.boxf, S.box_invf);
        // all walkers of the system rebuild together: their rebuild kernels
        // then run once, fully parallel, instead of on most steps
        if (dx * dx + dy * dy + dz * dz > S.half_skin2)
            for (int k = 0; k < S.w_count; ++k) d.rebuild[S.w_first + k] = 1;
    }
}

// atoms: the final B of the last step of a call
__global__ void k_finish(Dev d, int w0, int w1, int g0, int g1) {
    const int nthr = gridDim.x * blockDim.x;
    for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += nthr) {
        if (d.atom_of_slot[g] < 0) continue;
        const int w = d.slot_walker[g];
        const SysDev &S = d.sys[d.walk[w].sys];
        const unsigned long long *Fp = d.F + 3 * (size_t)g;
        const float hk = 0.5f * S.dt * d.im[g].x;
        float4 v = d.vv[g];
        v.x += hk * fix_to_float(Fp[0]);
        v.y += hk * fix_to_float(Fp[1]);
        v.z += hk * fix_to_float(Fp[2]);
        d.vv[g] = v;
    }
    if (blockIdx.x == 0)
        for (int w = w0 + threadIdx.x; w < w1; w += blockDim.x) d.pending[w] = 0;
}

// ---------------------------------------------------------------------------
// bonds (1/2 k (r - r0)^2), angles (1/2 k (theta - theta0)^2) and positional
// restraints (1/2 k |x - x0|^2); one thread per term
// ---------------------------------------------------------------------------
template <bool ENERGY>
__global__ void k_bonded(Dev d, int w0, int w1) {
    const int b0 = d.walk[w0].bo_off;
    const int b1 = d.walk[w1 - 1].bo_off + d.walk[w1 - 1].n_bo;
    const int nthr = gridDim.x * blockDim.x;
    for (int t = b0 + blockIdx.x * blockDim.x + threadIdx.x; t < b1; t += nthr) {
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
            const int gi = soa[ij.x], gj = soa[ij.y];
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
            const int gi = soa[ijk.x], gj = soa[ijk.y], gk = soa[ijk.z];
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
            const int gi = soa[ai];
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
}

// ---------------------------------------------------------------------------
// per walker: flat-bottom COM restraint, lambda-switched well, and the sum of
// the alchemical partials into s = dU/dlambda (fixed order: deterministic)
// ---------------------------------------------------------------------------
template <bool ENERGY>
__global__ void k_walker(Dev d, int w0) {
    const int w = w0 + blockIdx.x;
    const WalkerDev &W = d.walk[w];
    const SysDev &S = d.sys[W.sys];
    const int *soa = d.slot_of_atom + W.atom_base;
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ double red[8][32];
    __shared__ double sh_com[2][4];
    double lv, le, dlv, dle;
    lambda_path(d.lam[w], S.b_v, S.b_e, lv, le, dlv, dle);

    // ---- flat-bottom restraint on |COM_a - COM_b| ----
    if (S.n_fb_a > 0 && S.n_fb_b > 0) {
        for (int grp = 0; grp < 2; ++grp) {
            const int off = S.fb_off + (grp ? S.n_fb_a : 0);
            const int ng = grp ? S.n_fb_b : S.n_fb_a;
            const float4 r0 = d.xq[soa[d.fb_idx[off]]];
            double acc[4] = {0, 0, 0, 0};
            for (int k = tid; k < ng; k += nt) {
                const int a = d.fb_idx[off + k];
                const float4 xa = d.xq[soa[a]];
                const double m = 1.0 / (double)d.ap[S.atom_off + a].w;
                acc[0] += m * min_image(xa.x - r0.x, S.boxf, S.box_invf);
                acc[1] += m * min_image(xa.y - r0.y, S.boxf, S.box_invf);
                acc[2] += m * min_image(xa.z - r0.z, S.boxf, S.box_invf);
                acc[3] += m;
            }
            for (int c = 0; c < 4; ++c) {
                double v = warp_sum(acc[c]);
                if ((tid & 31) == 0) red[c][tid >> 5] = v;
            }
            __syncthreads();
            if (tid < 4) {
                double v = 0.0;
                for (int k = 0; k < (nt >> 5); ++k) v += red[tid][k];
                sh_com[grp][tid] = v;
            }
            __syncthreads();
            if (tid == 0) {
                sh_com[grp][0] = r0.x + sh_com[grp][0] / sh_com[grp][3];
                sh_com[grp][1] = r0.y + sh_com[grp][1] / sh_com[grp][3];
                sh_com[grp][2] = r0.z + sh_com[grp][2] / sh_com[grp][3];
            }
            __syncthreads();
        }
        double dv[3];
        for (int c = 0; c < 3; ++c) {
            double t = sh_com[0][c] - sh_com[1][c];
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
                const double mt = sh_com[grp][3];
                for (int k = tid; k < ng; k += nt) {
                    const int a = d.fb_idx[off + k];
                    const double wgt = (1.0 / (double)d.ap[S.atom_off + a].w) / mt;
                    add_force(d, soa[a], (float)(sgn * fmag * dv[0] * wgt), (float)(sgn * fmag * dv[1] * wgt),
                              (float)(sgn * fmag * dv[2] * wgt));
                }
            }
            if (ENERGY && tid == 0)
                atomicAdd((unsigned long long *)&d.eterm[N_ETERMS * w + 6],
                          (unsigned long long)__double2ll_rn(0.5 * S.fb_k * ex * ex * E_TO_FIX));
        }
    }

    // ---- lambda-switched harmonic well (uses lambda itself) ----
    double dl_dir = 0.0, e_lh = 0.0, dk1 = 0.0, d2k1 = 0.0;
    // ---- lambda-dependent distance restraint (Sec. 4.2): pairs kept at
    // least d_min = delta/2 (1 - cos 2 pi lambda) apart ----
    if (S.n_lr > 0) {
        const double lam = d.lam[w];
        const double dmin = 0.5 * S.lr_delta * (1.0 - cospi(2.0 * lam));
        const double ddmin = S.lr_delta * 3.14159265358979323846 * sinpi(2.0 * lam);
        for (int k = tid; k < S.n_lr; k += nt) {
            const int2 ab = d.lr_ij[S.lr_off + k];
            const int ga = soa[ab.x], gb = soa[ab.y];
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
    if (S.n_lh > 0) {
        const double lam = d.lam[w];
        const double kl = (1.0 - lam) * S.lh_k0 + lam * S.lh_k1;
        for (int k = tid; k < S.n_lh; k += nt) {
            const int a = d.lh_idx[S.lh_off + k];
            const int g = soa[a];
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
    {
        double v[4] = {dl_dir, e_lh, dk1, d2k1};
        __syncthreads();
        for (int c = 0; c < 4; ++c) {
            double t = warp_sum(v[c]);
            if ((tid & 31) == 0) red[c][tid >> 5] = t;
        }
        __syncthreads();
        if (tid == 0) {
            for (int c = 0; c < 4; ++c) {
                double t = 0.0;
                for (int k = 0; k < (nt >> 5); ++k) t += red[c][k];
                v[c] = t;
            }
            // ---- s = dU/dlambda: alchemical partials in atom order ----
            double sv = 0.0, se = 0.0, usc = 0.0, urf = 0.0;
            for (int r = 0; r < S.n_alch; ++r) {
                const double *o = d.alch_out + 4 * (size_t)(W.alch_base + r);
                sv += o[0];
                se += o[1];
                usc += o[2];
                urf += o[3];
            }
            d.s[w] = dlv * sv + dle * se + v[0];
            if (S.theta_stats || ENERGY) {
                double *th = d.wth + (size_t)w * 2 * d.P_max;
                for (int r = 0; r < S.n_alch; ++r) {
                    const double *o = d.alch_th + 6 * (size_t)(W.alch_base + r);
                    th[3 * r + 0] = o[0];
                    th[3 * r + 1] = o[1];
                    th[3 * r + 2] = o[2];
                    th[d.P_max + 3 * r + 0] = dlv * o[3];
                    th[d.P_max + 3 * r + 1] = dlv * o[4];
                    th[d.P_max + 3 * r + 2] = dle * o[5];
                }
                th[S.P - 1] = v[2];
                th[d.P_max + S.P - 1] = v[3];
            }
            if (ENERGY) {
                long long *et = d.eterm + N_ETERMS * w;
                atomicAdd((unsigned long long *)&et[2], (unsigned long long)__double2ll_rn(usc * E_TO_FIX));
                atomicAdd((unsigned long long *)&et[3], (unsigned long long)__double2ll_rn(urf * E_TO_FIX));
                atomicAdd((unsigned long long *)&et[6], (unsigned long long)__double2ll_rn(v[1] * E_TO_FIX));
                d.dl_direct[w] = v[0];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// ABF: fold the samples of a stage's walkers, merge every shared_freq steps,
// bias = min(1, n/n_full) * mean, final B of lambda; one block per stage.
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

__global__ void k_lambda(Dev d, int s0, int prime) {
    const StageDev &st = d.stage[s0 + blockIdx.x];
    const SysDev &S = d.sys[st.sys];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (!prime) {
        // fold each walker's sample into its own statistics (independent)
        for (int w = st.w0 + tid; w < st.w1; w += nt) {
            const int k = bin_of(d.lam[w], st);
            const size_t lk = (size_t)w * d.max_bins + k;
            const double sv = d.s[w];
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
                    d.th_d2[b] += th[d.P_max + p];
                    d.th_d[b] += th[p];
                    d.th_sd[b] += d.s[w] * th[p];
                }
            }
        }
        __syncthreads();
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
        __syncthreads();
    }
    for (int w = st.w0 + tid; w < st.w1; w += nt) {
        const double G = -d.s[w] + abf_bias(d, S, st, w);
        d.G[w] = G;
        if (!prime) {
            if (S.lambda_dynamics) d.plam[w] += 0.5 * S.dt_d * G;
            d.step[w] += 1ull;
            d.pending[w] = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_integrate(const Dev &d, const HostView &hv, int w0, int w1, cudaStream_t s) {
    const int g0 = hv.slot_off[w0], g1 = hv.slot_off[w1 - 1] + hv.slot_cap[w1 - 1];
    int blocks = (g1 - g0 + 255) / 256;
    blocks = blocks < 1 ? 1 : blocks;
    blocks = blocks > hv.n_sm * 8 ? hv.n_sm * 8 : blocks;
    k_integrate<<<blocks + 1, 256, 0, s>>>(d, w0, w1, g0, g1);
}

void launch_finish(const Dev &d, const HostView &hv, int w0, int w1, cudaStream_t s) {
    const int g0 = hv.slot_off[w0], g1 = hv.slot_off[w1 - 1] + hv.slot_cap[w1 - 1];
    int blocks = (g1 - g0 + 255) / 256;
    blocks = blocks < 1 ? 1 : (blocks > hv.n_sm * 8 ? hv.n_sm * 8 : blocks);
    k_finish<<<blocks, 256, 0, s>>>(d, w0, w1, g0, g1);
}

void launch_bonded(const Dev &d, const HostView &hv, int w0, int w1, bool energy, cudaStream_t s) {
    const int n = hv.bo_off[w1 - 1] + hv.n_bo[w1 - 1] - hv.bo_off[w0];
    if (n <= 0) return;
    int blocks = (n + 255) / 256;
    blocks = blocks > hv.n_sm * 8 ? hv.n_sm * 8 : blocks;
    if (energy) k_bonded<true><<<blocks, 256, 0, s>>>(d, w0, w1);
    else k_bonded<false><<<blocks, 256, 0, s>>>(d, w0, w1);
}

void launch_walker(const Dev &d, int w0, int w1, bool energy, cudaStream_t s) {
    if (energy) k_walker<true><<<w1 - w0, 256, 0, s>>>(d, w0);
    else k_walker<false><<<w1 - w0, 256, 0, s>>>(d, w0);
}

void launch_lambda(const Dev &d, int s0, int s1, bool prime, cudaStream_t s) {
    k_lambda<<<s1 - s0, 128, 0, s>>>(d, s0, prime ? 1 : 0);
}

}  // namespace labf
