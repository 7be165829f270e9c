/*
 * labf.h -- C ABI of the GB300 multiple-walker lambda-ABF engine.
 *
 * The engine advances many walkers of one or more systems with Langevin
 * lambda-dynamics under an Adaptive Biasing Force on lambda (arXiv
 * 2307.08006, Sec. 2.1-2.4).  Each walker carries atoms (x, v) and an
 * extended lambda particle (lambda, p_lambda).  One MD step evaluates the
 * alchemically scaled soft-core Lennard-Jones + reaction-field pair forces
 * and, in the same pair pass, the walker's dU/dlambda; it folds every
 * walker's dU/dlambda into the shared lambda-binned accumulator of its
 * stage (sum, sum of squares, count); it applies ramp * bin mean as the
 * bias on lambda; and it advances atoms and lambda with BAOAB.  The
 * accumulator's running mean integrated over lambda is Delta A (Sec. 2.3).
 *
 * The calls mirror the engine <-> Colvars contract of Sec. 3.2: parameters
 * are fixed once (la_create_system); each step the engine computes forces
 * and dU/dlambda at the current lambda, the bias is updated from the
 * accumulator and lambda is advanced (la_step_walkers); the free-energy
 * estimate is read back on demand (la_read_abf).
 *
 * Conventions for every call:
 *   - All calls are extern "C", return an int status (LA_OK = 0, negative
 *     LA_ERR_* on failure) and throw no C++ exception across the ABI.
 *   - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *     pointers are CUDA global memory owned by the caller.  The library
 *     never frees caller memory.
 *   - Device work is enqueued on the caller's stream (cudaStream_t passed as
 *     void*; NULL = the legacy default stream).  Calls marked
 *     "synchronising" wait for that stream before returning.
 *   - After an error, la_last_error(h) gives a message; a device-side error
 *     (list overflow, non-finite state, fixed-point overflow) is sticky:
 *     further stepping calls return LA_ERR_STATE until la_destroy.
 *
 * Units are the caller's (reduced LJ units, or nm, ps, amu, kJ/mol, e);
 * the engine only requires them to be consistent.
 */
#ifndef LABF_H
#define LABF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LA_OK 0
#define LA_ERR_INVALID_ARG (-1)
#define LA_ERR_BOX_TOO_SMALL (-2)   /* box edge < 2 (r_cut + skin) */
#define LA_ERR_CUDA (-3)
#define LA_ERR_UNSUPPORTED (-4)
#define LA_ERR_ARENA_TOO_SMALL (-5)
#define LA_ERR_LIST_OVERFLOW (-6)   /* a neighbour-list capacity was exceeded */
#define LA_ERR_NONFINITE (-7)       /* NaN/Inf appeared in positions or lambda */
#define LA_ERR_FIXED_OVERFLOW (-8)  /* a force exceeded the 64-bit fixed-point range */
#define LA_ERR_STATE (-9)           /* the handle is in a sticky error state */
#define LA_ERR_BAD_INDEX (-10)      /* range-checked builds (LA_CHECKS): an index read from a
                                       device list, cell or slot array was out of range */

/* ---- device status bits (la_sync / la_status) ---- */
#define LA_STATUS_LIST_OVERFLOW 0x1u
#define LA_STATUS_NONFINITE 0x2u
#define LA_STATUS_FIXED_OVERFLOW 0x4u
#define LA_STATUS_COLUMN_OVERFLOW 0x8u
#define LA_STATUS_ALCH_OVERFLOW 0x10u
#define LA_STATUS_BAD_INDEX 0x20u /* la_alch_pairs_static: alch_idx entry not an alchemical atom;
                                     range-checked builds: an index out of range */
#define LA_STATUS_BAD_PARAM 0x40u /* la_energy_forces_device: negative or non-finite epsilon, sigma, q */

/* ---- energy terms reported by la_energy_forces ---- */
#define LA_PAIR_VARIANTS 3
#define LA_MAX_WALKERS 256 /* walkers per handle, over all its systems */
#define LA_N_TERMS 7 /* LJ, RF, soft-core LJ, scaled RF, bond, angle, restraint */

/* ---- flags of la_energy_forces ---- */
#define LA_EF_REBUILD 0x1u      /* rebuild the neighbour lists first (positions were set) */
#define LA_EF_COUNT_PAIRS 0x2u  /* count in-cutoff pairs (returned by la_stats) */

typedef struct la_handle la_handle;

/*
 * One system: topology, force field, alchemical and ABF parameters, and the
 * initial state of its walkers.  All pointers are host memory, read during
 * la_query_sizes / la_create_system only (copied).
 *
 *   Force field (Sec. 3.1.2): pairs interact with Lennard-Jones
 *   (Lorentz-Berthelot mixing of per-atom sigma, epsilon) and reaction-field
 *   electrostatics coul*q_i*q_j*(1/r + k_rf r^2 - c_rf), both truncated at
 *   r_cut.  A pair with exactly one alchemical atom is scaled: soft-core LJ
 *   lambda_v^sc_n 4 eps (s^-2 - s^-1), s = sc_alpha (1-lambda_v)^sc_m +
 *   (r/sigma)^6 (integer powers sc_n, sc_m >= 1), and lambda_e times the
 *   RF term.  Pairs of two alchemical atoms, pairs in the same excl_group
 *   (>= 0) and pairs listed in excl_extra are excluded.  lambda -> (lambda_v, lambda_e) is the
 *   piecewise-linear path of Sec. 3.1.1 with breakpoints b_v, b_e.
 *   eps_rf <= 0 selects a conducting continuum.
 *
 *   Dynamics (Sec. 2.1, 2.2, Eq. lambda-abf; SI S1): BAOAB with collision
 *   rates gamma (atoms) and gamma_lambda (lambda), temperature kT, time step
 *   dt, lambda mass m_lambda.  lambda is reflected at its stage's walls.
 *   lambda_dynamics = 0 freezes lambda (fixed-lambda windows).
 *
 *   ABF (Sec. 2.3, 3.3, 2.4): n_stages stages, each with its own lambda
 *   interval [stage_lo, stage_hi] inside [0, 1], stage_bins >= 1 bins and
 *   stage_walkers >= 1 walkers (walkers are ordered by stage; at most
 *   LA_MAX_WALKERS = 256 walkers over all systems of a handle).  The bias is
 *   min(1, n_k / n_full) * (bin mean); walkers merge their samples into the
 *   shared statistics every shared_freq steps (shared_freq = 0: only when the
 *   host calls la_abf_import).  abf_on = 0 disables the bias.
 *
 *   Initial state: x0, v0 are [W][n_atoms][3] float32 (W = total walkers of
 *   the system), lam0 and plam0 are [W] double.  Philox streams are keyed by
 *   (seed, walker index within the system).
 */
typedef struct {
    int32_t n_atoms;
    double box; /* cubic box edge L */
    const double *mass, *charge, *sigma, *epsilon; /* [n_atoms] */
    const uint8_t *alch;                           /* [n_atoms] 1 = alchemical */
    const int32_t *excl_group;                     /* [n_atoms], -1 = none */
    const int32_t *excl_extra;                     /* [n_atoms][4], -1 padded */
    int32_t n_bonds;  const int32_t *bond_ij;   const double *bond_r0, *bond_k;
    int32_t n_angles; const int32_t *angle_ijk; const double *angle_t0, *angle_k;
    int32_t n_posres; const int32_t *posres_idx; const double *posres_x0; double posres_k;
    int32_t n_fb_a; const int32_t *fb_a; int32_t n_fb_b; const int32_t *fb_b;
    double fb_d0, fb_k;                            /* flat-bottom on |COM_a - COM_b| */
    int32_t n_lh; const int32_t *lh_idx; const double *lh_x0;
    double lh_k0, lh_k1; int32_t lh_dims;          /* 1/2 k(lambda) |x - x0|^2 */
    double r_cut, eps_rf, coul;
    double b_v, b_e, sc_alpha; int32_t sc_n, sc_m;
    double kT, dt, gamma, m_lambda, gamma_lambda, skin, n_full;
    int32_t shared_freq; uint32_t seed;
    int32_t lambda_dynamics, abf_on, theta_stats;
    int32_t n_stages;
    const double *stage_lo, *stage_hi;
    const int32_t *stage_bins, *stage_walkers;
    const float *x0, *v0;       /* [W][n_atoms][3] */
    const double *lam0, *plam0; /* [W] */
    /* lambda-dependent distance restraint (Sec. 4.2): each atom pair in
     * lr_ij ([n_lr][2]) gets 1/2 lr_k (d - d_min)^2 while d < d_min(lambda) =
     * lr_delta/2 (1 - cos 2 pi lambda), and contributes to dU/dlambda */
    int32_t n_lr; const int32_t *lr_ij; double lr_delta, lr_k;
} la_system_desc;

/* Engine options; zero-initialise for defaults. */
typedef struct {
    int32_t graph_steps;         /* MD steps captured per CUDA-graph replay (0: 10); < 0:
                                    no graph, one batched launch sequence per step (every
                                    list kernel is launched and returns early unless a
                                    walker must rebuild), e.g. for per-kernel profilers */
    int32_t autotune;            /* 1: pick pair-kernel launch shape by timing at create */
    double list_capacity_factor; /* >= 1 safety factor on list capacities (default 1.6) */
    int32_t pair_variant;        /* pair kernel when not autotuned, [0, LA_PAIR_VARIANTS):
                                    0 = 8 warps/CTA with 80 registers (default), 1 = 4
                                    warps/72, 2 = 4 warps/64.  All give identical
                                    results. */
    int32_t pair_ctas_per_sm;    /* pair grid in 8-warp CTA equivalents per SM (0 = 4) */
    int32_t chunk_entries;       /* cluster-pair entries per warp work item, a multiple of
                                    32 (0 = 32) */
    double prune_margin;         /* dynamic pruning of the batched step: tiles with no
                                    listed pair within r_cut + prune_margin are skipped
                                    until some atom of the system has moved 0.45
                                    prune_margin; then the next batched pair pass
                                    evaluates the listed tiles of all its walkers and
                                    prunes them again (so does the pass after a list
                                    rebuild).  0 (default), < 0 or >= skin = off.
                                    Results are identical either way. */
} la_options;

/*
 * la_query_sizes: bytes of device memory the engine needs for these systems
 * (one arena, 256-byte aligned).  Host-only; no device work.
 * Errors: LA_ERR_INVALID_ARG (bad counts, sizes or parameters),
 * LA_ERR_BOX_TOO_SMALL (L < 2 (r_cut + skin)).
 */
int la_query_sizes(const la_system_desc *sys, int n_sys, const la_options *opt,
                   size_t *arena_bytes);

/*
 * la_create_system: build an engine for n_sys systems (Sec. 3.2: parameters
 * initialised once).  `arena` is caller-owned device memory of at least
 * la_query_sizes bytes, 256-byte aligned; the engine carves all of its
 * device state out of it and never allocates device memory itself.  The
 * initial state is uploaded, neighbour lists are built and forces,
 * dU/dlambda and the lambda force are evaluated (no sample is folded).
 * Synchronising on `stream`.  On success *out owns host metadata and CUDA
 * graphs only.  Errors: LA_ERR_INVALID_ARG, LA_ERR_BOX_TOO_SMALL,
 * LA_ERR_ARENA_TOO_SMALL, LA_ERR_CUDA, LA_ERR_LIST_OVERFLOW.
 */
int la_create_system(const la_system_desc *sys, int n_sys, const la_options *opt, void *arena,
                     size_t arena_bytes, void *stream, la_handle **out);

/*
 * la_step_walkers: advance every walker of every system by n_steps BAOAB
 * steps with the ABF fold and bias each step (Eq. lambda-abf; Sec. 2.4 with
 * sharing every shared_freq steps), as one batched launch sequence per step
 * replayed from a CUDA graph.  Asynchronous: returns after enqueueing on
 * `stream`; it first checks the status word left by earlier calls and
 * returns LA_ERR_STATE (with la_last_error) if a device error was recorded.
 */
int la_step_walkers(la_handle *h, int64_t n_steps, void *stream);

/*
 * la_step_walkers_plain: the same n_steps, issued as one launch sequence per
 * walker and per phase without CUDA graphs (the one-walker-per-launch
 * form).  Results are identical to la_step_walkers.  Asynchronous.
 */
int la_step_walkers_plain(la_handle *h, int64_t n_steps, void *stream);

/*
 * la_read_abf: the accumulator of stage `stage` of system `sys` and its TI
 * read-out (Sec. 2.3): per bin k the sum, sum of squares and count of
 * dU/dlambda samples, grad[k] = sum/count (NaN for an empty bin), the
 * Riemann sum A[k] at the bin edges (A has n_bins + 1 entries, A[0] = 0),
 * *dA = A[n_bins], and *dA_se = w * sqrt(sum_k var_k / n_k), a naive
 * standard error that ignores time correlation.  Samples not yet merged
 * (shared_freq > 1) are not included.  Any output pointer may be NULL.
 * Host arrays, caller-owned.  Synchronising.  Returns LA_OK, or 1
 * (LA_WARN_EMPTY_BIN) when a bin is empty.
 */
#define LA_WARN_EMPTY_BIN 1
int la_read_abf(la_handle *h, int sys, int stage, double *sum, double *sumsq, int64_t *count,
                double *grad, double *A, double *dA, double *dA_se, void *stream);

/*
 * la_abf_export / la_abf_import: host-level sharing of the accumulator
 * between engines (walkers on other GPUs or processes; Sec. 2.4: walkers
 * periodically share their mean-force estimates).  Use with shared_freq = 0,
 * which disables the on-device merge: every walker then biases with the
 * shared statistics plus its own samples since the last exchange.  Engines
 * whose walkers cooperate must use distinct seeds (the Philox key is
 * (seed, walker index within the handle's system)), or their noise coincides.
 * la_abf_export fills host [n_bins] arrays with the stage's unmerged
 * statistics summed over its walkers in walker order (sum, sumsq: double;
 * count: int64).  la_abf_import adds host [n_bins] totals (normally the
 * rank-ordered sum of every engine's export, so that all engines keep
 * identical shared statistics) to the shared statistics, clears the stage's
 * unmerged statistics and re-evaluates the lambda force of every walker with
 * the new bias; it takes effect from the next step's first lambda half-kick.
 * Call both between la_step_walkers calls.  Errors: LA_ERR_INVALID_ARG for a
 * bad system/stage, a NULL pointer or a negative count (nothing is changed);
 * device errors as for la_step_walkers.  Both synchronising.
 */
int la_abf_export(la_handle *h, int sys, int stage, double *sum, double *sumsq, int64_t *count,
                  void *stream);
int la_abf_import(la_handle *h, int sys, int stage, const double *sum, const double *sumsq,
                  const int64_t *count, void *stream);

/*
 * la_energy_forces: energies and forces of one walker (global walker index)
 * at its current state (Sec. 3.2: the engine's gradient routine).
 * energy_terms (host, may be NULL): [LA_N_TERMS] doubles.
 * forces (device, may be NULL): [n_atoms][3] float32, -dU/dx.
 * dUdl (host, may be NULL): dU/dlambda.
 * dUdtheta, d2Udl_dtheta (host, may be NULL): [P] doubles with
 * P = 3 n_alch + 1: (eps, sigma, q) of each alchemical atom in index order,
 * then k1 of the lambda-switched well; dU/dtheta and d2U/dlambda dtheta.
 * flags: LA_EF_REBUILD to rebuild the lists first (needed after positions
 * were set by la_set_state), LA_EF_COUNT_PAIRS to count in-cutoff pairs.
 * The walker's stored force is refreshed as a side effect.  Synchronising.
 */
int la_energy_forces(la_handle *h, int walker, uint32_t flags, double *energy_terms,
                     float *forces, double *dUdl, double *dUdtheta, double *d2Udl_dtheta,
                     void *stream);

/*
 * la_energy_forces_device: the same evaluation with every input and output in
 * device memory and no host synchronisation (for the differentiation path:
 * U(x, lambda, theta) and its hand-written derivatives, north-star
 * extension; the paper does not differentiate with respect to force-field
 * parameters).  x (device [n_atoms][3] float32, atom order, or NULL: keep
 * the walker's positions) replaces the walker's positions and its lists are
 * rebuilt from them (recomputed, not stored); theta (device [n_alch][3]
 * double: epsilon, sigma, q of each alchemical atom in index order, or NULL)
 * replaces the system's alchemical parameters for all its walkers (the other
 * walkers are refreshed before their next use); lam (device double, or
 * NULL) replaces the walker's lambda.  out (device double, or NULL) receives
 * [LA_N_TERMS] energy terms, U, dU/dlambda, dU/dtheta [P] and
 * d2U/dlambda dtheta [P] (P = 3 n_alch + 1, the last entry k1 of the
 * lambda-switched well); forces (device [n_atoms][3] float32, or NULL)
 * receives -dU/dx.  Asynchronous on `stream`: a device error (including
 * LA_STATUS_BAD_PARAM for negative or non-finite epsilon or sigma, which
 * leaves those atoms' parameters unchanged) is reported by the next call.
 */
int la_energy_forces_device(la_handle *h, int walker, const float *x, const double *theta,
                            const double *lam, double *out, float *forces, void *stream);

/*
 * la_get_state / la_set_state: positions, velocities (host [n][3] float32),
 * lambda and p_lambda (host double) and the step counter of one walker, in
 * the system's atom order.  The step counter is the counter of the walker's
 * Philox streams (SI S1 BAOAB noise): setting it back repeats the noise of
 * that step.  After la_set_state the walker's lists and forces (no sample is
 * folded) are rebuilt once, for every walker set since, before the next call
 * that needs them (la_step_walkers[_plain], la_energy_forces, la_get_pairs,
 * la_time_kernels, la_autotune, la_abf_import, la_checkpoint_save), so that
 * setting all walkers costs one refresh.  Any pointer may be NULL (left
 * unchanged / not read).  If a copy fails part way, the walker may hold part
 * of the new state and the handle goes into the sticky error state.
 * Synchronising.
 */
int la_get_state(la_handle *h, int walker, float *x, float *v, double *lam, double *plam,
                 uint64_t *step, void *stream);
int la_set_state(la_handle *h, int walker, const float *x, const float *v, const double *lam,
                 const double *plam, const uint64_t *step, void *stream);

/*
 * la_get_states / la_set_states: the same for every walker at once, with one
 * synchronisation per call.  x and v (host float32) hold the walkers one
 * after another in handle order, walker w's [n_atoms][3] block starting at
 * 3 * (sum of n_atoms over walkers < w); lam, plam (host double) and step
 * (host uint64) hold one value per walker; any pointer may be NULL (left
 * unchanged / not read).  Only page-locked host buffers are copied by DMA
 * without intermediate waits; pageable buffers go through the driver's
 * staging, which waits for each copy.  After la_set_states every walker's
 * lists and forces are refreshed before the next call that needs them, as
 * after la_set_state (a failed copy leaves the handle in the sticky error
 * state).  Synchronising.
 */
int la_get_states(la_handle *h, float *x, float *v, double *lam, double *plam, uint64_t *step,
                  void *stream);
int la_set_states(la_handle *h, const float *x, const float *v, const double *lam, const double *plam,
                  const uint64_t *step, void *stream);

/*
 * la_checkpoint_save / la_checkpoint_load: the engine's complete state (every
 * walker's atoms in their current slot order, neighbour lists, pruning state,
 * forces, lambda particles, step counters, ABF accumulators shared and
 * unmerged, theta statistics, counters) as one host byte image, for exact
 * restarts (SI S1: runs are continued from saved states).  A run restored
 * from a checkpoint into an engine created from the same inputs and options
 * continues bit for bit as the run that saved it would have.
 *
 * la_checkpoint_save: *bytes receives the image size (a header plus the
 * state part of the arena, a few hundred MB for 16 walkers of 12 300 atoms);
 * with buf = NULL nothing else happens.  Otherwise buf (host, caller-owned,
 * cap bytes, page-locked for a fast copy) receives the image.  Refreshes
 * pending lists first (after la_set_state).  Errors: LA_ERR_INVALID_ARG when
 * cap is too small, LA_ERR_STATE after a device error.  Synchronising.
 *
 * la_checkpoint_load: replace the engine's state with an image.  The engine
 * must have been created from the same systems, run parameters and options
 * (the header's fingerprint of the layout and parameters and its
 * chunk_entries must match; LA_ERR_INVALID_ARG otherwise, with nothing
 * changed).  Clears a sticky error state if the image is clean.
 * Synchronising.
 */
int la_checkpoint_save(la_handle *h, void *buf, size_t cap, size_t *bytes, void *stream);
int la_checkpoint_load(la_handle *h, const void *buf, size_t bytes, void *stream);

/*
 * la_set_alch_params: replace (epsilon, sigma, charge) of the alchemical
 * atoms of system `sys` (host [n_alch][3] double, alchemical atoms in index
 * order) for the differentiation path; forces are re-evaluated.
 * Synchronising.
 */
int la_set_alch_params(la_handle *h, int sys, const double *theta, void *stream);

/*
 * la_read_theta: per-bin theta statistics of stage `stage` of system `sys`
 * (theta_stats = 1): sums of d2U/dlambda dtheta, of dU/dtheta and of
 * dU/dlambda * dU/dtheta, each host [n_bins][P] (may be NULL), and the
 * derivative of the stage's Delta A with respect to theta (host [P], may be
 * NULL): sum_k w [<d2U/dlambda dtheta>_k - Cov_k(dU/dlambda, dU/dtheta)/kT].
 * The paper does not differentiate Delta A; the covariance term is needed
 * because the lambda-conditional ensemble itself depends on theta.  All
 * samples folded so far count (merged or not).  Synchronising.  Returns
 * LA_WARN_EMPTY_BIN (NaN derivatives) when a bin is empty.
 */
int la_read_theta(la_handle *h, int sys, int stage, double *sum_d2, double *sum_d, double *sum_sd,
                  double *dA_dtheta, void *stream);

/*
 * la_get_pairs: expand the current neighbour list of one walker into atom
 * pairs (i < j, system atom indices) with kind 0 (normal) or 1 (one atom
 * alchemical), sorted by (i, j).  `pairs` is host [cap][2] int32, `kind`
 * host [cap] uint8; *count receives the total (may exceed cap).  Debug /
 * parity aid.  Synchronising.
 */
int la_get_pairs(la_handle *h, int walker, int32_t *pairs, uint8_t *kind, int64_t cap,
                 int64_t *count, void *stream);

/*
 * la_lambda_path: lambda -> {lambda_v, lambda_e, dlambda_v/dlambda,
 * dlambda_e/dlambda} (Sec. 3.1.1) evaluated by the engine's device code for
 * n values with breakpoints b_v, b_e, staged through the handle's I/O
 * buffer (n up to a few thousand; LA_ERR_INVALID_ARG beyond).
 * lam: host [n]; out: host [n][4].  Synchronising.
 */
int la_lambda_path(la_handle *h, const double *lam, int n, double b_v, double b_e, double *out,
                   void *stream);

/*
 * la_sync: wait for `stream`, then return the status as an LA_ERR_* code
 * (LA_OK if clean); *status_bits (may be NULL) receives LA_STATUS_* bits.
 */
int la_sync(la_handle *h, void *stream, uint32_t *status_bits);

/*
 * la_stats: counters since creation.  out (host, may be NULL) receives
 *   [0] MD steps taken, [1] list rebuilds (summed over walkers),
 *   [2] kernel launches issued by the engine (graph nodes counted per replay),
 *   [3] in-cutoff normal pairs counted by the last LA_EF_COUNT_PAIRS call,
 *   [4] in-cutoff alchemical pairs counted by that call,
 *   [5] cluster-pair entries in the current lists (all walkers),
 *   [6] 8 x 4 atom-pair tiles the batched step evaluates (all walkers, after
 *       the last dynamic pruning); each tile is one warp-wide evaluation of
 *       32 candidate pairs,
 *   [7] re-pruning passes of the batched step (summed over walkers) after a
 *       displacement trigger.
 * Synchronising.
 */
#define LA_N_STATS 8
int la_stats(la_handle *h, int64_t *out, void *stream);

/*
 * la_time_kernels: run n_steps batched steps outside the graph with CUDA
 * events between the launches on `stream`, in the order and with the
 * conditions of the graph's step: the integrator, the gate kernel, the list
 * kernels only on steps where some walker must rebuild (the host reads the
 * walkers' rebuild flags after the gate, as the graph's conditional node
 * does on the device), and the fused pair launch.  ms_out (host
 * [LA_N_KERNELS]) receives the mean device milliseconds per MD step of each
 * class (so that integrate + rebuild + pairs is the step's kernel time, the
 * list kernels averaged over the steps at the rebuild rate met), and
 * launches_out (host [LA_N_KERNELS], may be NULL) the launch counts.  In the
 * batched step the bonded terms, the walker terms and the lambda update run
 * inside the pair launch, so their classes read 0.  Synchronising.
 */
#define LA_N_KERNELS 6 /* integrate, rebuild (gate + list kernels when due), pairs, bonded, walker, lambda */
int la_time_kernels(la_handle *h, int n_steps, float *ms_out, int64_t *launches_out, void *stream);

/*
 * la_autotune: choose the pair kernel's launch shape (variant, grid, work-item
 * size) by timing repeated pair-kernel launches on the current neighbour
 * lists, e.g. after equilibration, when the lists differ from those of the
 * starting structure.  The state does not change: forces are restored bit
 * for bit afterwards, and every shape gives identical results.  The CUDA
 * graph is re-captured.  la_create_system with autotune = 1 does the same
 * at creation (reusing an earlier result for the same system shape).
 * Synchronising.
 */
int la_autotune(la_handle *h, void *stream);

/*
 * la_fp_peak: measured fused-multiply-add rate of this GPU (the current
 * device), in TFLOP/s (an FMA counts 2): fp64 = 0 for FP32 (the CUDA-core
 * peak the pair pass's roofline is taken against), 1 for FP64.  Runs
 * independent FMA chains on every SM for about `seconds` (0 < seconds <= 10)
 * of device time after a warm-up, timed with CUDA events on `stream`.  A
 * measurement aid for the roofline (the paper has no counterpart).
 * Synchronising.  Errors: LA_ERR_INVALID_ARG, LA_ERR_CUDA.
 */
int la_fp_peak(int fp64, double seconds, double *tflops, void *stream);

/* la_autotune_report: text describing the chosen launch shapes (static buffer). */
const char *la_autotune_report(la_handle *h);

/* la_last_error: message of the last failing call on h (static per handle). */
const char *la_last_error(la_handle *h);

/* la_destroy: free host metadata and CUDA graphs; never touches the arena. */
int la_destroy(la_handle *h);

/*
 * la_alch_pairs_static: the alchemical part of the pair pass for one
 * configuration, for callers that cannot allocate device memory.  (The
 * paper has no counterpart; this is a deployment aid.)
 *
 * Who needs it: code that runs as a plugin inside another program that owns
 * the GPU's memory (for example an MD engine that hands a force routine its
 * own buffers and forbids further allocations), and code that must keep a
 * fixed device footprint declared up front.  Such callers cannot create an
 * engine (la_create_system needs a caller-allocated arena), so this entry
 * point needs no handle and calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * It evaluates, for every alchemical atom a and every non-alchemical atom b
 * of another exclusion group within r_cut (minimum image in a cubic box of
 * edge `box`), the soft-core LJ lambda_v^sc_n 4 eps (s^-2 - s^-1),
 * s = sc_alpha (1 - lambda_v)^sc_m + (r/sigma)^6 (Lorentz-Berthelot mixing),
 * plus lambda_e times the reaction-field term coul q_a q_b (1/r + k_rf r^2 -
 * c_rf), with (lambda_v, lambda_e) from lam by the b_v / b_e path.  Pairs
 * are scanned directly (no neighbour list).  Only excl_group exclusions
 * apply (no per-atom extra exclusion lists).
 *
 * Inputs (device memory, caller-owned): x [n_atoms][3] float32, q, sigma,
 * epsilon [n_atoms] float32, alch [n_atoms] uint8 (1 = alchemical),
 * excl_group [n_atoms] int32 (-1 = none), alch_idx [n_alch] int32 (the
 * indices of the alchemical atoms, ascending, each in [0, n_atoms), flagged
 * in alch and listed once).  sc_n, sc_m >= 1.
 * Outputs (device memory, caller-owned, overwritten): forces [n_atoms][3]
 * float32 = minus the gradient of these pair terms; out [6] double =
 * {dU/dlambda, dU/dlambda_v, dU/dlambda_e, soft-core LJ energy,
 * lambda_e * RF energy, status}.  status is 0, or the LA_STATUS_* bits of
 * what went wrong on the device: LA_STATUS_BAD_INDEX (an alch_idx entry
 * outside [0, n_atoms) or not flagged alchemical: that atom is skipped),
 * LA_STATUS_NONFINITE (a non-finite distance or force: the pair is
 * skipped), LA_STATUS_FIXED_OVERFLOW (a force component of 2^30 or more,
 * beyond the fixed-point accumulators: skipped).  Any non-zero status
 * means the other outputs are incomplete.
 *
 * Scratch: one file-scope static device array of 3 * LA_STATIC_MAX_ATOMS
 * 64-bit force accumulators plus 4 * LA_STATIC_MAX_ALCH doubles (about
 * 3.2 MB), held by every GPU that loads the library until the process
 * exits.  Each call clears the part it uses before using it.  All calls on
 * a device share that one array, so calls whose GPU work overlaps (on
 * different streams, or from different threads) race and corrupt each
 * other's results; serialise them.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (with that device current); make that first call before any stream
 * capture begins.
 *
 * Errors: LA_ERR_INVALID_ARG for NULL pointers, non-positive sizes or box,
 * sc_n < 1 or sc_m < 1, n_atoms > LA_STATIC_MAX_ATOMS or n_alch > LA_STATIC_MAX_ALCH (the message
 * of la_static_last_error names the limit); LA_ERR_CUDA if the set-up or a
 * launch fails.  Asynchronous on `stream`.
 */
#define LA_STATIC_MAX_ATOMS 131072
#define LA_STATIC_MAX_ALCH 1024
int la_alch_pairs_static(int n_atoms, const float *x, const float *q, const float *sigma,
                         const float *epsilon, const uint8_t *alch, const int32_t *excl_group,
                         int n_alch, const int32_t *alch_idx, double box, double r_cut,
                         double eps_rf, double coul, double lam, double b_v, double b_e,
                         double sc_alpha, int sc_n, int sc_m, float *forces, double *out,
                         void *stream);

/* la_static_last_error: message of the last failing la_alch_pairs_static call
 * on this thread. */
const char *la_static_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LABF_H */
