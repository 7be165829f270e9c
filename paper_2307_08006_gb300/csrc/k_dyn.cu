// k_dyn.cu -- BAOAB of atoms and lambda, bonded and restraint terms, the
// per-walker dU/dlambda sum, and the ABF fold / bias / TI helpers.
//
// Step order (Eq. lambda-abf; BAOAB as in SI Sec. S1), per MD step:
//   k_integrate : [finish B of the previous step] B A O A for atoms and lambda
//   (rebuild)   : neighbour lists if any atom moved more than skin/2
//   k_pairs     : forces, dU/dlambda partials           (k_pairs.cu)
//   k_bonded    : bonds, angles, positional restraints
//   k_walker    : restraints on walker level, dU/dlambda sum
//   k_lambda    : fold samples, bias, final B of lambda
// and once at the end of a call k_finish applies the atoms' final B.  The
// batched step runs the last four as one launch (k_pairs.cu, fused form);
// the bodies shared by both forms are in labf_dyn.cuh.
#include "labf_dyn.cuh"
#include "labf_internal.cuh"
#include "labf_launch.h"

namespace labf {

// ---------------------------------------------------------------------------
// atoms: BAOA (with the previous step's final B when pending), lambda: BAOA
// ---------------------------------------------------------------------------
__global__ void k_integrate(Dev d, int w0, int w1, int g0, int g1) {
    const int nthr = gridDim.x * blockDim.x;
    // lambda particles (FP64): the first w1-w0 threads of block 0, which is
    // scheduled first, so that this work overlaps the atoms'
    if (blockIdx.x == 0) {
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
        // every per-slot load is issued before the first branch (padding
        // slots are readable too), so they are all in flight together
        const int a = d.atom_of_slot[g];
        const int w = d.slot_walker[g];
        unsigned long long *Fp = d.F + 3 * (size_t)g;
        const unsigned long long f0 = Fp[0], f1 = Fp[1], f2 = Fp[2];
        const float2 im = d.im[g];
        float4 v = d.vv[g];
        const float4 x0 = d.xq[g];
        float4 x = x0;
        const float4 r = d.xref[g];
        if (a < 0) continue;
        const WalkerDev &W = d.walk[w];
        const SysDev &S = d.sys[W.sys];
        float fx = fix_to_float(f0), fy = fix_to_float(f1), fz = fix_to_float(f2);
        if (fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))) > FIX_LIMIT) set_status(d, LA_STATUS_FIXED_OVERFLOW);
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
        float dx = min_image(x.x - r.x, S.boxf, S.box_invf);
        float dy = min_image(x.y - r.y, S.boxf, S.box_invf);
        float dz = min_image(x.z - r.z, S.boxf, S.box_invf);
        // all walkers of the system rebuild together: their rebuild kernels
        // then run once, fully parallel, instead of on most steps
        const float disp2 = dx * dx + dy * dy + dz * dz;
        if (disp2 > S.half_skin2)
            for (int k = 0; k < S.w_count; ++k) d.rebuild[S.w_first + k] = 1;
        else if (disp2 > S.near_skin2)
            for (int k = 0; k < S.w_count; ++k) d.near[S.w_first + k] = 1;
        // the same for the pruned tiles of the batched step; all walkers of the
        // system re-prune together, so that a pair launch runs either the
        // pruning form of the item loop or the common one.  The positions this
        // step starts from are the new reference when the previous step's pair
        // pass re-pruned the walker (it ran with the step counter one below the
        // current one).
        if (S.prune_disp2 > 0.f) {
            float4 rp;
            if (d.prune_now[w] == d.step[w]) {
                rp = x0;
                d.xprune[g] = x0;
            } else {
                rp = d.xprune[g];
            }
            dx = min_image(x.x - rp.x, S.boxf, S.box_invf);
            dy = min_image(x.y - rp.y, S.boxf, S.box_invf);
            dz = min_image(x.z - rp.z, S.boxf, S.box_invf);
            if (dx * dx + dy * dy + dz * dz > S.prune_disp2)
                for (int k = 0; k < S.w_count; ++k) d.prune[S.w_first + k] = 1;
        }
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

// bonded terms, one thread per term
template <bool ENERGY>
__global__ void k_bonded(Dev d, int w0, int w1) {
    const int b0 = d.walk[w0].bo_off;
    const int b1 = d.walk[w1 - 1].bo_off + d.walk[w1 - 1].n_bo;
    const int nthr = gridDim.x * blockDim.x;
    for (int t = b0 + blockIdx.x * blockDim.x + threadIdx.x; t < b1; t += nthr) bonded_term<ENERGY>(d, t, w0, w1);
}

// walker terms, one warp per walker
template <bool ENERGY>
__global__ void k_walker(Dev d, int w0, int w1) {
    const int w = w0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w < w1) walker_work<ENERGY>(d, w, threadIdx.x & 31);
}

// ABF fold / bias / final B of lambda, one block per stage
__global__ void k_lambda(Dev d, int s0, int prime) {
    lambda_work<false>(d, s0 + blockIdx.x, prime, threadIdx.x, blockDim.x);
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
    const int blocks = (w1 - w0 + 3) / 4;
    if (energy) k_walker<true><<<blocks, 128, 0, s>>>(d, w0, w1);
    else k_walker<false><<<blocks, 128, 0, s>>>(d, w0, w1);
}

void launch_lambda(const Dev &d, int s0, int s1, bool prime, cudaStream_t s) {
    k_lambda<<<s1 - s0, 128, 0, s>>>(d, s0, prime ? 1 : 0);
}

}  // namespace labf
