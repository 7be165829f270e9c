// labf_launch.h -- host-side launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include "labf_internal.cuh"

#define LA_MAX_WALKERS_PER_LAUNCH LA_MAX_WALKERS

namespace labf {

// Host copies of the per-walker offsets the launchers size grids with.
struct HostView {
    int n_walkers = 0, n_sm = 0, pair_blocks = 0, ncs = 1;
    int pair_variant = 0;  // 0: 8 warps/CTA, 80 regs; 1: 4 warps, 72; 2: 4 warps, 64
    const int *slot_off = nullptr, *slot_cap = nullptr, *sc_cap = nullptr, *n_cols = nullptr;
    const int *alch_base = nullptr, *n_alch = nullptr, *item_cap = nullptr;
    const int *bo_off = nullptr, *n_bo = nullptr;
};

void launch_integrate(const Dev &d, const HostView &hv, int w0, int w1, cudaStream_t s);
void launch_finish(const Dev &d, const HostView &hv, int w0, int w1, cudaStream_t s);
// batched: the batched step's chain (fresh lists are pruned by its pair pass)
void launch_rebuild(const Dev &d, const HostView &hv, int w0, int w1, cudaStream_t s, bool batched = false);
void launch_items(const Dev &d, const HostView &hv, int w0, int w1, cudaStream_t s);
// conditional: also set the graph's conditional handle (false outside graphs)
void launch_gate(const Dev &d, int w0, int w1, cudaGraphConditionalHandle handle, bool conditional,
                 cudaStream_t s);
int rebuild_kernel_count(const HostView &hv, int w0, int w1);
// rebuild coalescing of the one-walker-per-launch form (the batched step's
// gate does the same)
void launch_coalesce(const Dev &d, int w0, int w1, cudaStream_t s);
void launch_pairs(const Dev &d, const HostView &hv, int w0, int w1, bool energy, cudaStream_t s);
// pairs + bonded + walker terms + lambda update of all walkers in one launch
void launch_pairs_fused(const Dev &d, const HostView &hv, int n_stages, cudaStream_t s);
void launch_bonded(const Dev &d, const HostView &hv, int w0, int w1, bool energy, cudaStream_t s);
void launch_walker(const Dev &d, int w0, int w1, bool energy, cudaStream_t s);
void launch_lambda(const Dev &d, int s0, int s1, bool prime, cudaStream_t s);
void launch_state_io(const Dev &d, int w, int n, float *x, float *v, bool to_slots, cudaStream_t s);
void launch_forces_out(const Dev &d, int w, int n, float *out, cudaStream_t s);
void launch_lambda_path(const double *lam, int n, double bv, double be, double *out, cudaStream_t s);
void launch_positions_in(const Dev &d, int w, int n, const float *x, cudaStream_t s);
void launch_alch_params_in(const Dev &d, int sys, int n_alch, const double *theta, cudaStream_t s);
void launch_ef_out(const Dev &d, int w, int P, double *out, cudaStream_t s);

}  // namespace labf
