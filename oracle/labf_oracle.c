/*
 * labf_oracle.c -- FP64 CPU oracle for the lambda-ABF multiple-walker step
 * (Lagardere, Hedin, Henin et al., arXiv 2307.08006).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the
 * benchmark's CPU-baseline leg.  It is deliberately plain: O(N^2) pair loops
 * with the minimum-image convention, textbook formulas, no lists, no
 * blocking, no fused or reordered arithmetic beyond what each definition
 * states.  Build with -ffp-contract=off so that no multiply-add is fused.
 *
 * Passages followed (paper section / equation / table):
 *   lambda path ................ Sec. 3.1.1 and Fig. "alch-path"; SI Table S1
 *   soft-core LJ ............... Sec. 3.1.2 (scaling of Lennard-Jones by lambda_v);
 *                                the paper prints no formula: Beutler form read
 *   electrostatics ............. Sec. 3.1.2 (linear scaling by lambda_e); reaction
 *                                field stands in for PME
 *   Langevin lambda-dynamics ... Sec. 2.1, Eq. (lambdadyn-Langevin-process);
 *                                reflecting walls on lambda (Sec. 2.1)
 *   BAOAB ...................... SI Sec. S1 (BAOAB, 1 fs)
 *   ABF on lambda .............. Sec. 2.3, Eq. (lambda-abf); ramp: Sec. 3.3
 *   multiple walkers ........... Sec. 2.4 (periodic sharing of the mean force)
 *   Riemann-sum TI ............. Sec. 2.3 (free energy by integration)
 *
 * Parity pins (tests/test_oracle_*.py): SI Table S1 values; Philox
 * known-answer vectors; textbook LJ at lambda_v = 1; U = 0 at lambda_v = 0;
 * RF U(r_c) = 0 and F(r_c) = 0 for a conducting continuum; central finite
 * differences of U in x, lambda and theta; brute-force and constructed
 * boundary cases for the integer pair set; BAOAB's exact harmonic
 * configurational variance; the closed-form free energy of a
 * lambda-switched harmonic well and its derivative in k1; Newton's third
 * law and translation invariance of the pair forces.
 */
#include "labf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */

/* minimum-image displacement of one component in a cubic box */
static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ */
/* lambda -> (lambda_v, lambda_e): Sec. 3.1.1, Fig. alch-path, Table S1 */
/* ------------------------------------------------------------------ */
/* lambda_v rises linearly from 0 at lambda = 0 to 1 at lambda = b_v and stays
 * at 1 beyond; lambda_e is 0 up to lambda = b_e and rises linearly to 1 at
 * lambda = 1.  Slopes at the kinks are one-sided: d lambda_v / d lambda = 0
 * at lambda = b_v (the "lambda_v = 1 for lambda >= b_v" branch) and
 * d lambda_e / d lambda = 0 at lambda = b_e ("lambda_e = 0 for lambda <= b_e").
 * out = {lambda_v, lambda_e, d lambda_v/d lambda, d lambda_e/d lambda}. */
void or_lambda_path(double lam, double b_v, double b_e, double out[4]) {
    double lv, le, dlv, dle;
    if (lam >= b_v) {
        lv = 1.0;
        dlv = 0.0;
    } else {
        lv = lam / b_v;
        dlv = 1.0 / b_v;
    }
    if (lam <= b_e) {
        le = 0.0;
        dle = 0.0;
    } else {
        le = (lam - b_e) / (1.0 - b_e);
        dle = 1.0 / (1.0 - b_e);
    }
    out[0] = lv;
    out[1] = le;
    out[2] = dlv;
    out[3] = dle;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published  */
/* description: ten rounds of two 32x32->64 multiplies with the key bumped */
/* by the golden-ratio Weyl constants between rounds.                     */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Four standard normals for (walker, step, idx, tag): counter =
 * {idx, step_lo, step_hi, tag}, key = {seed, walker}.  Each pair of 32-bit
 * outputs gives u1 = (a>>8 + 1) 2^-24 in (0,1] and u2 = (b>>8) 2^-24 in [0,1),
 * and Box-Muller gives sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2). */
void or_normals4(uint32_t seed, uint32_t walker, uint64_t step, uint32_t idx, uint32_t tag,
                 double z[4]) {
    uint32_t ctr[4] = {idx, (uint32_t)step, (uint32_t)(step >> 32), tag};
    uint32_t key[2] = {seed, walker};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    for (int k = 0; k < 2; ++k) {
        double u1 = ((double)(r[2 * k] >> 8) + 1.0) * (1.0 / 16777216.0);
        double u2 = (double)(r[2 * k + 1] >> 8) * (1.0 / 16777216.0);
        double rad = sqrt(-2.0 * log(u1));
        double th = 2.0 * M_PI * u2;
        z[2 * k] = rad * cos(th);
        z[2 * k + 1] = rad * sin(th);
    }
}

/* ------------------------------------------------------------------ */
/* Integer pair set (bit-exact definition of the neighbour list)        */
/* ------------------------------------------------------------------ */
/* u = floor(frac(x * L^-1) * 2^24), with x * L^-1 one correctly rounded FP64
 * product and u = 2^24 folded to 0. */
void or_quantize(int n, const float *x, double box_inv, uint32_t *u) {
    for (int i = 0; i < 3 * n; ++i) {
        double t = (double)x[i] * box_inv;
        double f = t - floor(t);
        double s = floor(f * 16777216.0);
        uint32_t q = (uint32_t)s;
        if (q >= 16777216u) q = 0u;
        u[i] = q;
    }
}

/* R = floor((r_list L^-1)^2 2^48): pairs with integer squared distance D < R
 * are listed (ties D == R are not). */
int64_t or_list_threshold(double r_list, double box_inv) {
    double a = r_list * box_inv;
    double a2 = a * a;
    return (int64_t)floor(a2 * 281474976710656.0);
}

/* minimum-image component on the 2^24 torus, in [-2^23, 2^23) */
static int64_t torus_delta(uint32_t a, uint32_t b) {
    int64_t d = ((int64_t)a - (int64_t)b + 8388608) & 16777215;
    return d - 8388608;
}

static int or_excluded(const or_system *sys, int i, int j) {
    if (sys->excl_group[i] >= 0 && sys->excl_group[i] == sys->excl_group[j]) return 1;
    for (int k = 0; k < 4; ++k) {
        if (sys->excl_extra[4 * i + k] == j) return 1;
        if (sys->excl_extra[4 * j + k] == i) return 1;
    }
    if (sys->alch[i] && sys->alch[j]) return 1; /* intra-solute pairs are excluded */
    return 0;
}

/* All unordered pairs i<j, not excluded, with D < R.  kind = 0 for a normal
 * pair, 1 when exactly one atom is alchemical.  Returns the number of pairs;
 * at most cap are written. */
int64_t or_pair_set(const or_system *sys, const float *x, double box_inv, int64_t R,
                    int32_t *pairs, uint8_t *kind, int64_t cap) {
    int n = sys->n;
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    or_quantize(n, x, box_inv, u);
    int64_t cnt = 0;
    for (int i = 0; i < n; ++i) {
        for (int j = i + 1; j < n; ++j) {
            if (or_excluded(sys, i, j)) continue;
            int64_t dx = torus_delta(u[3 * i], u[3 * j]);
            int64_t dy = torus_delta(u[3 * i + 1], u[3 * j + 1]);
            int64_t dz = torus_delta(u[3 * i + 2], u[3 * j + 2]);
            int64_t D = dx * dx + dy * dy + dz * dz;
            if (D < R) {
                if (cnt < cap) {
                    pairs[2 * cnt] = i;
                    pairs[2 * cnt + 1] = j;
                    kind[cnt] = (uint8_t)((sys->alch[i] ? 1 : 0) + (sys->alch[j] ? 1 : 0));
                }
                ++cnt;
            }
        }
    }
    free(u);
    return cnt;
}

/* The pairs of or_pair_set that involve at least one atom flagged in
 * rows[n] (the same definition, visited only for flagged atoms, so that
 * very large systems can be checked on a sample of atoms).  Output in the
 * same (i, j) order as or_pair_set. */
int64_t or_pair_set_rows(const or_system *sys, const float *x, double box_inv, int64_t R, const uint8_t *rows,
                         int32_t *pairs, uint8_t *kind, int64_t cap) {
    int n = sys->n;
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    or_quantize(n, x, box_inv, u);
    int64_t cnt = 0;
    for (int i = 0; i < n; ++i) {
        for (int j = i + 1; j < n; ++j) {
            if (!rows[i] && !rows[j]) continue;
            if (or_excluded(sys, i, j)) continue;
            int64_t dx = torus_delta(u[3 * i], u[3 * j]);
            int64_t dy = torus_delta(u[3 * i + 1], u[3 * j + 1]);
            int64_t dz = torus_delta(u[3 * i + 2], u[3 * j + 2]);
            int64_t D = dx * dx + dy * dy + dz * dz;
            if (D < R) {
                if (cnt < cap) {
                    pairs[2 * cnt] = i;
                    pairs[2 * cnt + 1] = j;
                    kind[cnt] = (uint8_t)((sys->alch[i] ? 1 : 0) + (sys->alch[j] ? 1 : 0));
                }
                ++cnt;
            }
        }
    }
    free(u);
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Energies, forces, dU/dlambda, dU/dtheta                              */
/* ------------------------------------------------------------------ */
int or_n_theta(const or_system *sys) {
    int na = 0;
    for (int i = 0; i < sys->n; ++i) na += sys->alch[i] ? 1 : 0;
    return 3 * na + 1;
}

/* Reaction-field constants for cutoff rc and continuum permittivity eps_rf:
 * k_rf = (eps_rf - 1) / ((2 eps_rf + 1) rc^3), c_rf = 1/rc + k_rf rc^2;
 * eps_rf -> infinity gives k_rf = 1 / (2 rc^3). */
static void rf_constants(double rc, double eps_rf, double *krf, double *crf) {
    if (eps_rf <= 0.0)
        *krf = 1.0 / (2.0 * rc * rc * rc);
    else
        *krf = (eps_rf - 1.0) / ((2.0 * eps_rf + 1.0) * rc * rc * rc);
    *crf = 1.0 / rc + (*krf) * rc * rc;
}

/* x: [n][3] positions; F: [n][3] forces (= -dU/dx);
 * terms: LJ, RF, sc-LJ, sc-RF, bond, angle, restraint;
 * dl = {dU/dlambda_v, dU/dlambda_e, dU/dlambda from terms that use lambda itself};
 * dth / d2th: [P] dU/dtheta and d2U/dlambda dtheta, theta = (eps_a, sigma_a, q_a)
 * for each alchemical atom a in index order, then k1. */
static void energy_forces_impl(const or_system *sys, const double *x, double lam,
                               double terms[OR_N_TERMS], double *F, double dl[3], double *dUdl,
                               double *dth, double *d2th, const uint8_t *mask);

void or_energy_forces(const or_system *sys, const double *x, double lam,
                      double terms[OR_N_TERMS], double *F, double dl[3], double *dUdl,
                      double *dth, double *d2th) {
    energy_forces_impl(sys, x, lam, terms, F, dl, dUdl, dth, d2th, NULL);
}

/* Same, but nonbonded pairs are visited only when one atom is selected by
 * mask or alchemical: the forces on selected atoms, dU/dlambda and the theta
 * derivatives are complete; the other forces and the energy terms are not.
 * For sampled checks of systems too large for the full O(N^2) pass. */
void or_energy_forces_masked(const or_system *sys, const double *x, double lam, const uint8_t *mask,
                             double terms[OR_N_TERMS], double *F, double dl[3], double *dUdl,
                             double *dth, double *d2th) {
    energy_forces_impl(sys, x, lam, terms, F, dl, dUdl, dth, d2th, mask);
}

static void energy_forces_impl(const or_system *sys, const double *x, double lam,
                               double terms[OR_N_TERMS], double *F, double dl[3], double *dUdl,
                               double *dth, double *d2th, const uint8_t *mask) {
    const int n = sys->n;
    const double L = sys->box;
    double path[4];
    or_lambda_path(lam, sys->b_v, sys->b_e, path);
    const double lv = path[0], le = path[1], dlv = path[2], dle = path[3];
    const int P = or_n_theta(sys);
    double krf, crf;
    rf_constants(sys->r_cut, sys->eps_rf, &krf, &crf);
    const double rc2 = sys->r_cut * sys->r_cut;

    for (int t = 0; t < OR_N_TERMS; ++t) terms[t] = 0.0;
    for (int i = 0; i < 3 * n; ++i) F[i] = 0.0;
    double dUdlv = 0.0, dUdle = 0.0, dUdl_direct = 0.0;
    /* theta derivatives split by which lambda factor they carry */
    double *dth_v = (double *)calloc((size_t)P, sizeof(double)); /* d2U/dlv dtheta */
    double *dth_e = (double *)calloc((size_t)P, sizeof(double)); /* d2U/dle dtheta */
    for (int p = 0; p < P; ++p) dth[p] = 0.0;
    int *alch_rank = (int *)malloc(sizeof(int) * (size_t)n);
    {
        int r = 0;
        for (int i = 0; i < n; ++i) alch_rank[i] = sys->alch[i] ? r++ : -1;
    }

    /* ---- nonbonded pairs, O(N^2) with the minimum image ---- */
    for (int i = 0; i < n; ++i) {
        for (int j = i + 1; j < n; ++j) {
            if (mask && !mask[i] && !mask[j] && !sys->alch[i] && !sys->alch[j]) continue;
            if (or_excluded(sys, i, j)) continue;
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = min_image(x[3 * i + c] - x[3 * j + c], L);
            double r2 = dot3(d, d);
            if (r2 >= rc2) continue; /* plain truncation at r_c */
            double r = sqrt(r2);
            double sig = 0.5 * (sys->sigma[i] + sys->sigma[j]);     /* Lorentz */
            double eps = sqrt(sys->epsilon[i] * sys->epsilon[j]); /* Berthelot */
            double qq = sys->coul * sys->charge[i] * sys->charge[j];
            double rf_u = qq * (1.0 / r + krf * r2 - crf);
            double rf_f = qq * (1.0 / (r2 * r) - 2.0 * krf); /* -(dU/dr)/r */
            int one_alch = (sys->alch[i] ? 1 : 0) + (sys->alch[j] ? 1 : 0);
            double fscal; /* F_i = fscal * d, F_j = -fscal * d */
            if (one_alch == 0) {
                double sr2 = sig * sig / r2;
                double sr6 = sr2 * sr2 * sr2;
                double sr12 = sr6 * sr6;
                double lj_u = 4.0 * eps * (sr12 - sr6);
                double lj_f = 4.0 * eps * (12.0 * sr12 - 6.0 * sr6) / r2;
                terms[0] += lj_u;
                terms[1] += rf_u;
                fscal = lj_f + rf_f;
            } else {
                /* soft-core LJ: s = alpha (1-lv)^m + (r/sig)^6,
                   U = lv^n 4 eps (s^-2 - s^-1) */
                const double alpha = sys->sc_alpha;
                const int nn = sys->sc_n, mm = sys->sc_m;
                double rho6 = 0.0, s = 0.0, g = 0.0, g1 = 0.0, g2 = 0.0;
                double lvn = pow(lv, nn), dlvn = (double)nn * pow(lv, nn - 1);
                double ds_dlv = -(double)mm * alpha * pow(1.0 - lv, mm - 1);
                double sc_u = 0.0, sc_f = 0.0, sc_dlv = 0.0;
                if (eps > 0.0) {
                    double q2 = r2 / (sig * sig);
                    rho6 = q2 * q2 * q2;
                    s = alpha * pow(1.0 - lv, mm) + rho6;
                    g = 1.0 / (s * s) - 1.0 / s;
                    g1 = -2.0 / (s * s * s) + 1.0 / (s * s);
                    g2 = 6.0 / (s * s * s * s) - 2.0 / (s * s * s);
                    sc_u = lvn * 4.0 * eps * g;
                    /* dU/dr = lvn 4 eps g1 * 6 rho6 / r  ->  -(dU/dr)/r */
                    sc_f = -lvn * 4.0 * eps * g1 * 6.0 * rho6 / r2;
                    sc_dlv = dlvn * 4.0 * eps * g + lvn * 4.0 * eps * g1 * ds_dlv;
                }
                terms[2] += sc_u;
                terms[3] += le * rf_u;
                dUdlv += sc_dlv;
                dUdle += rf_u;
                fscal = sc_f + le * rf_f;
                /* theta derivatives for the alchemical member a of the pair */
                int a = sys->alch[i] ? i : j, b = sys->alch[i] ? j : i;
                int ra = alch_rank[a];
                double qb = sys->coul * sys->charge[b];
                double rf_shape = 1.0 / r + krf * r2 - crf;
                if (eps > 0.0 && sys->epsilon[a] > 0.0) {
                    double de = eps / (2.0 * sys->epsilon[a]);  /* d eps_ab / d eps_a */
                    dth[3 * ra + 0] += lvn * 4.0 * g * de;
                    dth_v[3 * ra + 0] += (dlvn * 4.0 * g + lvn * 4.0 * g1 * ds_dlv) * de;
                }
                if (eps > 0.0) {
                    double ds_dsig = -6.0 * rho6 / sig; /* d s / d sigma_ab */
                    /* d sigma_ab / d sigma_a = 1/2 */
                    dth[3 * ra + 1] += lvn * 4.0 * eps * g1 * ds_dsig * 0.5;
                    dth_v[3 * ra + 1] +=
                        (dlvn * 4.0 * eps * g1 * ds_dsig + lvn * 4.0 * eps * g2 * ds_dsig * ds_dlv) *
                        0.5;
                }
                dth[3 * ra + 2] += le * qb * rf_shape;
                dth_e[3 * ra + 2] += qb * rf_shape;
            }
            for (int c = 0; c < 3; ++c) {
                F[3 * i + c] += fscal * d[c];
                F[3 * j + c] -= fscal * d[c];
            }
        }
    }

    /* ---- harmonic bonds: U = 1/2 k (r - r0)^2 ---- */
    for (int b = 0; b < sys->n_bonds; ++b) {
        int i = sys->bond_ij[2 * b], j = sys->bond_ij[2 * b + 1];
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = min_image(x[3 * i + c] - x[3 * j + c], L);
        double r = sqrt(dot3(d, d));
        double dr = r - sys->bond_r0[b];
        terms[4] += 0.5 * sys->bond_k[b] * dr * dr;
        double fs = -sys->bond_k[b] * dr / r;
        for (int c = 0; c < 3; ++c) {
            F[3 * i + c] += fs * d[c];
            F[3 * j + c] -= fs * d[c];
        }
    }

    /* ---- harmonic angles: U = 1/2 k (theta - theta0)^2, vertex j ---- */
    for (int a = 0; a < sys->n_angles; ++a) {
        int i = sys->angle_ijk[3 * a], j = sys->angle_ijk[3 * a + 1], k = sys->angle_ijk[3 * a + 2];
        double u[3], w[3];
        for (int c = 0; c < 3; ++c) {
            u[c] = min_image(x[3 * i + c] - x[3 * j + c], L);
            w[c] = min_image(x[3 * k + c] - x[3 * j + c], L);
        }
        double nu = sqrt(dot3(u, u)), nw = sqrt(dot3(w, w));
        double cs = dot3(u, w) / (nu * nw);
        if (cs > 1.0) cs = 1.0;
        if (cs < -1.0) cs = -1.0;
        double th = acos(cs);
        double dth_ = th - sys->angle_t0[a];
        terms[5] += 0.5 * sys->angle_k[a] * dth_ * dth_;
        double dUdth = sys->angle_k[a] * dth_;
        double sn = sqrt(1.0 - cs * cs);
        /* d theta / d u = -(1/sin) (w/(|u||w|) - cos u/|u|^2) */
        for (int c = 0; c < 3; ++c) {
            double dcos_du = w[c] / (nu * nw) - cs * u[c] / (nu * nu);
            double dcos_dw = u[c] / (nu * nw) - cs * w[c] / (nw * nw);
            double fi = dUdth / sn * dcos_du;
            double fk = dUdth / sn * dcos_dw;
            F[3 * i + c] += fi;
            F[3 * k + c] += fk;
            F[3 * j + c] -= fi + fk;
        }
    }

    /* ---- positional restraints: U = 1/2 k |x - x0|^2 ---- */
    for (int p = 0; p < sys->n_posres; ++p) {
        int i = sys->posres_idx[p];
        for (int c = 0; c < 3; ++c) {
            double d = min_image(x[3 * i + c] - sys->posres_x0[3 * p + c], L);
            terms[6] += 0.5 * sys->posres_k * d * d;
            F[3 * i + c] -= sys->posres_k * d;
        }
    }

    /* ---- flat-bottom restraint on the distance of two centres of mass ---- */
    if (sys->n_fb_a > 0 && sys->n_fb_b > 0) {
        double com[2][3], mt[2];
        const int32_t *grp[2] = {sys->fb_a, sys->fb_b};
        int ng[2] = {sys->n_fb_a, sys->n_fb_b};
        for (int g = 0; g < 2; ++g) {
            int a0 = grp[g][0];
            double acc[3] = {0, 0, 0};
            mt[g] = 0.0;
            for (int k = 0; k < ng[g]; ++k) {
                int a = grp[g][k];
                double m = sys->mass[a];
                mt[g] += m;
                for (int c = 0; c < 3; ++c) acc[c] += m * min_image(x[3 * a + c] - x[3 * a0 + c], L);
            }
            for (int c = 0; c < 3; ++c) com[g][c] = x[3 * a0 + c] + acc[c] / mt[g];
        }
        double dv[3];
        for (int c = 0; c < 3; ++c) dv[c] = min_image(com[0][c] - com[1][c], L);
        double dd = sqrt(dot3(dv, dv));
        if (dd > sys->fb_d0) {
            double ex = dd - sys->fb_d0;
            terms[6] += 0.5 * sys->fb_k * ex * ex;
            double fmag = sys->fb_k * ex / dd; /* -dU/d(dv) = -fmag * dv */
            for (int g = 0; g < 2; ++g) {
                double sgn = g == 0 ? -1.0 : 1.0;
                for (int k = 0; k < ng[g]; ++k) {
                    int a = grp[g][k];
                    double w = sys->mass[a] / mt[g];
                    for (int c = 0; c < 3; ++c) F[3 * a + c] += sgn * fmag * dv[c] * w;
                }
            }
        }
    }

    /* ---- lambda-switched harmonic well (uses lambda itself) ---- */
    double dk1 = 0.0, d2k1 = 0.0;
    if (sys->n_lh > 0) {
        double kl = (1.0 - lam) * sys->lh_k0 + lam * sys->lh_k1;
        for (int p = 0; p < sys->n_lh; ++p) {
            int i = sys->lh_idx[p];
            double r2 = 0.0;
            for (int c = 0; c < sys->lh_dims; ++c) {
                double d = min_image(x[3 * i + c] - sys->lh_x0[3 * p + c], L);
                r2 += d * d;
                F[3 * i + c] -= kl * d;
            }
            terms[6] += 0.5 * kl * r2;
            dUdl_direct += 0.5 * (sys->lh_k1 - sys->lh_k0) * r2;
            dk1 += 0.5 * lam * r2;
            d2k1 += 0.5 * r2;
        }
    }
    dth[P - 1] = dk1;

    /* ---- lambda-dependent distance restraint (Sec. 4.2): the pair is kept
       at least d_min(lambda) = delta/2 (1 - cos 2 pi lambda) apart ---- */
    if (sys->n_lr > 0) {
        double dmin = 0.5 * sys->lr_delta * (1.0 - cos(2.0 * M_PI * lam));
        double ddmin = sys->lr_delta * M_PI * sin(2.0 * M_PI * lam); /* d d_min / d lambda */
        for (int p = 0; p < sys->n_lr; ++p) {
            int a = sys->lr_ij[2 * p], b = sys->lr_ij[2 * p + 1];
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = min_image(x[3 * a + c] - x[3 * b + c], L);
            double r = sqrt(dot3(d, d));
            if (r >= dmin) continue;
            double ex = r - dmin; /* negative */
            terms[6] += 0.5 * sys->lr_k * ex * ex;
            dUdl_direct += -sys->lr_k * ex * ddmin;
            double fs = -sys->lr_k * ex / r; /* F_a = fs * d */
            for (int c = 0; c < 3; ++c) {
                F[3 * a + c] += fs * d[c];
                F[3 * b + c] -= fs * d[c];
            }
        }
    }

    dl[0] = dUdlv;
    dl[1] = dUdle;
    dl[2] = dUdl_direct;
    *dUdl = dlv * dUdlv + dle * dUdle + dUdl_direct;
    for (int p = 0; p < P; ++p) d2th[p] = dlv * dth_v[p] + dle * dth_e[p];
    d2th[P - 1] = d2k1;
    free(dth_v);
    free(dth_e);
    free(alch_rank);
}

/* ------------------------------------------------------------------ */
/* ABF accumulator, bias, and the BAOAB step of atoms and lambda        */
/* ------------------------------------------------------------------ */
/* bin k = floor((lam - lo) / w), w = (hi - lo) / nb, clamped to [0, nb-1] */
int or_bin(double lam, double lo, double hi, int nb) {
    double w = (hi - lo) / (double)nb;
    int k = (int)floor((lam - lo) / w);
    if (k < 0) k = 0;
    if (k > nb - 1) k = nb - 1;
    return k;
}

static int stage_offset(const or_run_params *run, int stage) {
    int off = 0;
    for (int s = 0; s < stage; ++s) off += run->stage_bins[s];
    return off;
}

static int max_bins(const or_run_params *run) {
    int m = 0;
    for (int s = 0; s < run->n_stages; ++s)
        if (run->stage_bins[s] > m) m = run->stage_bins[s];
    return m;
}

/* ABF bias on lambda, Eq. (lambda-abf): + ramp * A'_t(lambda) with A'_t the
 * running bin mean of dU/dlambda and ramp = min(1, n_k / n_full) (Sec. 3.3);
 * an empty bin gives no bias.  The walker sees the shared statistics plus its
 * own samples since the last merge. */
static double abf_bias(const or_run_params *run, const or_state *st, int w) {
    if (!run->abf_on) return 0.0;
    int stage = st->walker_stage[w];
    int nb = run->stage_bins[stage];
    int k = or_bin(st->lam[w], run->stage_lo[stage], run->stage_hi[stage], nb);
    int off = stage_offset(run, stage);
    int mb = max_bins(run);
    double sum = st->abf_sum[off + k] + st->dl_sum[(size_t)w * mb + k];
    double cnt = (double)(st->abf_count[off + k] + st->dl_count[(size_t)w * mb + k]);
    if (cnt <= 0.0) return 0.0;
    double ramp = cnt / run->n_full;
    if (ramp > 1.0) ramp = 1.0;
    return ramp * sum / cnt;
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* thread count for the per-walker loops (independent walkers only) */
static int g_threads = 1;
void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int or_get_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void evaluate_walker(const or_system *sys, or_state *st, int w, int P) {
    double terms[OR_N_TERMS], dl[3];
    size_t n3 = 3 * (size_t)sys->n;
    or_energy_forces(sys, st->x + w * n3, st->lam[w], terms, st->F + w * n3, dl, &st->s[w],
                     st->dth + (size_t)w * P, st->d2th + (size_t)w * P);
}

/* Forces and dU/dlambda at the current state, and G = -dU/dlambda + bias,
 * without adding any sample to the accumulator. */
void or_prime(const or_system *sys, const or_run_params *run, or_state *st) {
    int P = or_n_theta(sys);
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
    for (int w = 0; w < st->n_walkers; ++w) evaluate_walker(sys, st, w, P);
    for (int w = 0; w < st->n_walkers; ++w) st->G[w] = -st->s[w] + abf_bias(run, st, w);
}

/* reflecting walls at lo and hi (Sec. 2.1): mirror the position, flip p */
static void reflect(double *lam, double *p, double lo, double hi) {
    for (;;) {
        if (*lam < lo) {
            *lam = 2.0 * lo - *lam;
            *p = -*p;
        } else if (*lam > hi) {
            *lam = 2.0 * hi - *lam;
            *p = -*p;
        } else {
            break;
        }
    }
}

/* n_steps of BAOAB for every walker (atoms and lambda), Eq. (lambda-abf):
 *   B: p += dt/2 F          (lambda: p_lam += dt/2 G)
 *   A: x += dt/2 p/m        (lambda reflected at the stage walls)
 *   O: p = c p + sqrt((1-c^2) m kT) xi,  c = exp(-gamma dt)
 *   A: x += dt/2 p/m        (reflected; atoms wrapped into [0, L))
 *   evaluate F and s = dU/dlambda at the new state, for all walkers
 *   fold every walker's s into its stage's bins in walker order (merging
 *   walker-local statistics every shared_freq steps, Sec. 2.4)
 *   G = -s + ramp * mean of the bin after the fold
 *   B: p += dt/2 F, p_lam += dt/2 G
 * The atom state is held as velocities v = p/m. */
void or_run(const or_system *sys, const or_run_params *run, or_state *st, int n_steps) {
    const int n = sys->n;
    const size_t n3 = 3 * (size_t)n;
    const double L = sys->box, dt = run->dt, kT = run->kT;
    const double c_at = exp(-run->gamma * dt);
    const double c_lm = exp(-run->gamma_lambda * dt);
    const int P = or_n_theta(sys);
    const int mb = max_bins(run);
    for (int it = 0; it < n_steps; ++it) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int w = 0; w < st->n_walkers; ++w) {
            double *x = st->x + w * n3, *v = st->v + w * n3, *F = st->F + w * n3;
            uint64_t step = st->step[w];
            int stage = st->walker_stage[w];
            double lo = run->stage_lo[stage], hi = run->stage_hi[stage];
            /* B */
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt * F[3 * i + c] / sys->mass[i];
            if (run->lambda_dynamics) st->plam[w] += 0.5 * dt * st->G[w];
            /* A */
            for (int i = 0; i < 3 * n; ++i) x[i] += 0.5 * dt * v[i];
            if (run->lambda_dynamics) {
                st->lam[w] += 0.5 * dt * st->plam[w] / run->m_lambda;
                reflect(&st->lam[w], &st->plam[w], lo, hi);
            }
            /* O */
            for (int i = 0; i < n; ++i) {
                double z[4];
                or_normals4(run->seed, (uint32_t)w, step, (uint32_t)i, 0u, z);
                double sd = sqrt((1.0 - c_at * c_at) * kT / sys->mass[i]);
                for (int c = 0; c < 3; ++c) v[3 * i + c] = c_at * v[3 * i + c] + sd * z[c];
            }
            if (run->lambda_dynamics) {
                double z[4];
                or_normals4(run->seed, (uint32_t)w, step, 0u, 1u, z);
                double sd = sqrt((1.0 - c_lm * c_lm) * run->m_lambda * kT);
                st->plam[w] = c_lm * st->plam[w] + sd * z[0];
            }
            /* A */
            for (int i = 0; i < 3 * n; ++i) {
                x[i] += 0.5 * dt * v[i];
                x[i] -= L * floor(x[i] / L);
            }
            if (run->lambda_dynamics) {
                st->lam[w] += 0.5 * dt * st->plam[w] / run->m_lambda;
                reflect(&st->lam[w], &st->plam[w], lo, hi);
            }
            st->step[w] = step + 1;
        }
        /* forces and samples at the new state */
#pragma omp parallel for schedule(dynamic) num_threads(g_threads)
        for (int w = 0; w < st->n_walkers; ++w) evaluate_walker(sys, st, w, P);
        /* fold, in walker order, into walker-local statistics */
        for (int w = 0; w < st->n_walkers; ++w) {
            int stage = st->walker_stage[w];
            int nb = run->stage_bins[stage];
            int k = or_bin(st->lam[w], run->stage_lo[stage], run->stage_hi[stage], nb);
            double sv = st->s[w];
            st->dl_sum[(size_t)w * mb + k] += sv;
            st->dl_sumsq[(size_t)w * mb + k] += sv * sv;
            st->dl_count[(size_t)w * mb + k] += 1;
            if (run->theta_stats) {
                int off = stage_offset(run, stage);
                for (int p = 0; p < P; ++p) {
                    double d = st->dth[(size_t)w * P + p];
                    st->th_d2[(size_t)(off + k) * P + p] += st->d2th[(size_t)w * P + p];
                    st->th_d[(size_t)(off + k) * P + p] += d;
                    st->th_sd[(size_t)(off + k) * P + p] += sv * d;
                }
            }
        }
        /* merge walker-local statistics into the shared ones every K steps */
        int K = run->shared_freq > 0 ? run->shared_freq : 1;
        if (st->step[0] % (uint64_t)K == 0) {
            for (int w = 0; w < st->n_walkers; ++w) {
                int stage = st->walker_stage[w];
                int off = stage_offset(run, stage);
                for (int k = 0; k < run->stage_bins[stage]; ++k) {
                    size_t lk = (size_t)w * mb + k;
                    st->abf_sum[off + k] += st->dl_sum[lk];
                    st->abf_sumsq[off + k] += st->dl_sumsq[lk];
                    st->abf_count[off + k] += st->dl_count[lk];
                    st->dl_sum[lk] = 0.0;
                    st->dl_sumsq[lk] = 0.0;
                    st->dl_count[lk] = 0;
                }
            }
        }
        /* generalized force on lambda with the updated bias, and the final B */
        for (int w = 0; w < st->n_walkers; ++w) {
            st->G[w] = -st->s[w] + abf_bias(run, st, w);
            double *v = st->v + w * n3, *F = st->F + w * n3;
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt * F[3 * i + c] / sys->mass[i];
            if (run->lambda_dynamics) st->plam[w] += 0.5 * dt * st->G[w];
        }
    }
}

/* ------------------------------------------------------------------ */
/* TI read-out (Sec. 2.3): the bin mean estimates the bin-averaged        */
/* gradient; A at the bin edges is its Riemann sum, Delta A the total.    */
/* ------------------------------------------------------------------ */
void or_ti(const double *sum, const int64_t *count, int nb, double lo, double hi,
           double *grad, double *A, double *dA) {
    double w = (hi - lo) / (double)nb;
    A[0] = 0.0;
    for (int k = 0; k < nb; ++k) {
        grad[k] = count[k] > 0 ? sum[k] / (double)count[k] : NAN;
        A[k + 1] = A[k] + w * grad[k];
    }
    *dA = A[nb];
}

/* Derivative of Delta A in theta (not in the paper): for each bin,
 * <d2U/dlambda dtheta> - beta Cov(dU/dlambda, dU/dtheta), integrated by the
 * same Riemann sum.  The covariance term is required because the
 * lambda-conditional ensemble itself depends on theta. */
void or_theta_gradient(const double *sum, const int64_t *count, const double *th_d2,
                       const double *th_d, const double *th_sd, int nb, double lo,
                       double hi, int P, double kT, double *dA_dtheta) {
    double w = (hi - lo) / (double)nb;
    for (int p = 0; p < P; ++p) dA_dtheta[p] = 0.0;
    for (int k = 0; k < nb; ++k) {
        if (count[k] <= 0) {
            for (int p = 0; p < P; ++p) dA_dtheta[p] = NAN;
            continue;
        }
        double cnt = (double)count[k];
        double ms = sum[k] / cnt;
        for (int p = 0; p < P; ++p) {
            double m2 = th_d2[(size_t)k * P + p] / cnt;
            double md = th_d[(size_t)k * P + p] / cnt;
            double msd = th_sd[(size_t)k * P + p] / cnt;
            dA_dtheta[p] += w * (m2 - (msd - ms * md) / kT);
        }
    }
}
