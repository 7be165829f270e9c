/*
 * labf_oracle.h -- interface of the FP64 CPU oracle for the lambda-ABF
 * multiple-walker step (arXiv 2307.08006).
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, O(N^2) statement
 * of what the GPU engine computes.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no header,
 * table, constant or helper with the CUDA engine; the two are compared only
 * through their outputs on identical seeded inputs.
 *
 * Units are whatever the caller uses consistently (reduced LJ units, or
 * nm / ps / amu / kJ mol^-1 / e).  All arrays are row-major, caller-owned.
 */
#ifndef LABF_ORACLE_H
#define LABF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of energy terms reported by or_energy_forces. */
#define OR_N_TERMS 7 /* LJ, RF, sc-LJ, sc-RF, bond, angle, restraint */

typedef struct {
    int n;                      /* atoms */
    double box;                 /* cubic box edge L */
    const double *mass;         /* [n] */
    const double *charge;       /* [n] */
    const double *sigma;        /* [n]  LJ sigma_i */
    const double *epsilon;      /* [n]  LJ epsilon_i */
    const uint8_t *alch;        /* [n]  1 = alchemical (perturbed) atom */
    const int32_t *excl_group;  /* [n]  equal ids >= 0 do not interact (nonbonded) */
    const int32_t *excl_extra;  /* [n*4] further excluded partners, -1 padded */
    int n_bonds;  const int32_t *bond_ij;   const double *bond_r0, *bond_k;
    int n_angles; const int32_t *angle_ijk; const double *angle_t0, *angle_k;
    int n_posres; const int32_t *posres_idx; const double *posres_x0; double posres_k;
    /* flat-bottom restraint between the centres of mass of groups A and B */
    int n_fb_a; const int32_t *fb_a; int n_fb_b; const int32_t *fb_b; double fb_d0, fb_k;
    /* lambda-switched harmonic well: U = 1/2 ((1-lam) k0 + lam k1) |x - x0|^2 over
       the first lh_dims Cartesian components */
    int n_lh; const int32_t *lh_idx; const double *lh_x0; double lh_k0, lh_k1; int lh_dims;
    /* lambda-dependent distance restraint (Sec. 4.2): for each atom pair,
       1/2 k (d - d_min)^2 when d < d_min(lambda) = delta/2 (1 - cos 2 pi lambda) */
    int n_lr; const int32_t *lr_ij; double lr_delta, lr_k;
    double r_cut, eps_rf, coul; /* eps_rf <= 0 means a conducting (infinite) continuum */
    double b_v, b_e;            /* lambda -> (lambda_v, lambda_e) breakpoints */
    double sc_alpha; int sc_n, sc_m;
} or_system;

typedef struct {
    double kT, dt, gamma;            /* atoms: collision rate gamma */
    double m_lambda, gamma_lambda;   /* extended lambda particle */
    int lambda_dynamics;             /* 0: lambda frozen (fixed-lambda windows) */
    int abf_on;                      /* 0: no adaptive bias */
    double n_full;                   /* ramp: min(1, n_k / n_full) */
    int shared_freq;                 /* walkers merge bin statistics every K steps */
    uint32_t seed;
    int n_stages;
    const double *stage_lo, *stage_hi;
    const int32_t *stage_bins;
    int theta_stats;                 /* accumulate per-bin theta statistics */
} or_run_params;

typedef struct {
    int n_walkers;
    const int32_t *walker_stage;     /* [W] */
    double *x, *v;                   /* [W][n][3] */
    double *lam, *plam;              /* [W] */
    uint64_t *step;                  /* [W] */
    double *F;                       /* [W][n][3] force at the current state */
    double *G;                       /* [W] generalized force on lambda (incl. bias) */
    double *s;                       /* [W] last dU/dlambda */
    double *dth, *d2th;              /* [W][P] last dU/dtheta, d2U/dlambda dtheta */
    double *abf_sum, *abf_sumsq;     /* [sum of stage bins] shared statistics */
    int64_t *abf_count;
    double *dl_sum, *dl_sumsq;       /* [W][max_bins] walker-local deltas (K > 1) */
    int64_t *dl_count;
    double *th_d2, *th_d, *th_sd;    /* [sum of stage bins][P] */
} or_state;

/* Number of theta parameters: (eps, sigma, q) per alchemical atom, plus k1. */
int or_n_theta(const or_system *sys);

void or_lambda_path(double lam, double b_v, double b_e, double out[4]);

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_normals4(uint32_t seed, uint32_t walker, uint64_t step, uint32_t idx,
                 uint32_t tag, double z[4]);

void or_quantize(int n, const float *x, double box_inv, uint32_t *u);
int64_t or_list_threshold(double r_list, double box_inv);
int64_t or_pair_set(const or_system *sys, const float *x, double box_inv, int64_t R,
                    int32_t *pairs, uint8_t *kind, int64_t cap);
int64_t or_pair_set_rows(const or_system *sys, const float *x, double box_inv, int64_t R, const uint8_t *rows,
                         int32_t *pairs, uint8_t *kind, int64_t cap);

void or_energy_forces(const or_system *sys, const double *x, double lam,
                      double terms[OR_N_TERMS], double *F, double dl[3], double *dUdl,
                      double *dth, double *d2th);

void or_energy_forces_masked(const or_system *sys, const double *x, double lam, const uint8_t *mask,
                             double terms[OR_N_TERMS], double *F, double dl[3], double *dUdl,
                             double *dth, double *d2th);

void or_set_threads(int n);
int or_get_max_threads(void);

int or_bin(double lam, double lo, double hi, int nb);
void or_prime(const or_system *sys, const or_run_params *run, or_state *st);
void or_run(const or_system *sys, const or_run_params *run, or_state *st, int n_steps);
void or_ti(const double *sum, const int64_t *count, int nb, double lo, double hi,
           double *grad, double *A, double *dA);
void or_theta_gradient(const double *sum, const int64_t *count, const double *th_d2,
                       const double *th_d, const double *th_sd, int nb, double lo,
                       double hi, int P, double kT, double *dA_dtheta);

#ifdef __cplusplus
}
#endif
#endif
