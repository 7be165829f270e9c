// k_io.cu -- state and force transfer between the slot layout and the
// system's atom order, and the lambda-path evaluator.
#include "labf_internal.cuh"
#include "labf_launch.h"

namespace labf {

// to_slots = 0: x, v (atom order) <- slots;  1: slots <- x, v
__global__ void k_state_io(Dev d, int w, int n, float *x, float *v, int to_slots) {
    const WalkerDev &W = d.walk[w];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = checked_slot(d, d.slot_of_atom[W.atom_base + i]);
        if (to_slots) {
            float4 xq = d.xq[g];
            xq.x = x[3 * i];
            xq.y = x[3 * i + 1];
            xq.z = x[3 * i + 2];
            d.xq[g] = xq;
            d.vv[g] = make_float4(v[3 * i], v[3 * i + 1], v[3 * i + 2], 0.f);
        } else {
            const float4 xq = d.xq[g], vv = d.vv[g];
            x[3 * i] = xq.x;
            x[3 * i + 1] = xq.y;
            x[3 * i + 2] = xq.z;
            v[3 * i] = vv.x;
            v[3 * i + 1] = vv.y;
            v[3 * i + 2] = vv.z;
        }
    }
}

__global__ void k_forces_out(Dev d, int w, int n, float *out) {
    const WalkerDev &W = d.walk[w];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = checked_slot(d, d.slot_of_atom[W.atom_base + i]);
        const unsigned long long *F = d.F + 3 * (size_t)g;
        out[3 * i] = fix_to_float(F[0]);
        out[3 * i + 1] = fix_to_float(F[1]);
        out[3 * i + 2] = fix_to_float(F[2]);
        if (fabsf(out[3 * i]) > FIX_LIMIT || fabsf(out[3 * i + 1]) > FIX_LIMIT || fabsf(out[3 * i + 2]) > FIX_LIMIT)
            set_status(d, LA_STATUS_FIXED_OVERFLOW);
    }
}

__global__ void k_lambda_path(const double *lam, int n, double bv, double be, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double lv, le, dlv, dle;
        lambda_path(lam[i], bv, be, lv, le, dlv, dle);
        out[4 * i] = lv;
        out[4 * i + 1] = le;
        out[4 * i + 2] = dlv;
        out[4 * i + 3] = dle;
    }
}

// positions of walker w from a device array in atom order; the walker's
// lists are rebuilt before its next force evaluation
__global__ void k_positions_in(Dev d, int w, int n, const float *x) {
    const WalkerDev &W = d.walk[w];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = checked_slot(d, d.slot_of_atom[W.atom_base + i]);
        float4 xq = d.xq[g];
        xq.x = x[3 * i];
        xq.y = x[3 * i + 1];
        xq.z = x[3 * i + 2];
        d.xq[g] = xq;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d.rebuild[w] = 1;
}

// (epsilon, sigma, q) of the alchemical atoms of system `sys` from a device
// array; every walker of the system rebuilds (the per-slot copies of the
// parameters are refreshed there).  Negative or non-finite epsilon or sigma:
// the atom keeps its parameters and LA_STATUS_BAD_PARAM is set.
__global__ void k_alch_params_in(Dev d, int sys, const double *theta) {
    const SysDev &S = d.sys[sys];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < S.n_alch; r += gridDim.x * blockDim.x) {
        const double eps = theta[3 * r], sig = theta[3 * r + 1], q = theta[3 * r + 2];
        if (!(eps >= 0.0) || !(sig >= 0.0) || !(eps < 1e30) || !(sig < 1e30) || !(fabs(q) < 1e30)) {
            set_status(d, LA_STATUS_BAD_PARAM);
            continue;
        }
        const int a = d.alch_atoms[S.alch_off + r];
        float4 p = d.aparam_mut[S.atom_off + a];
        p.x = (float)(q * (double)S.sqrt_coul);
        p.y = (float)(0.5 * sig);
        p.z = (float)(2.0 * sqrt(eps));
        d.aparam_mut[S.atom_off + a] = p;
    }
    if (blockIdx.x == 0)
        for (int w = S.w_first + threadIdx.x; w < S.w_first + S.w_count; w += blockDim.x) d.rebuild[w] = 1;
}

// energies and derivatives of walker w into a device array: [0, LA_N_TERMS)
// the energy terms, then U, dU/dlambda, dU/dtheta [P], d2U/dlambda dtheta [P]
__global__ void k_ef_out(Dev d, int w, int P, double *out) {
    const int t = threadIdx.x;
    if (t == 0) {
        double u = 0.0;
        for (int k = 0; k < LA_N_TERMS; ++k) {
            const double e = (double)d.eterm[N_ETERMS * w + k] / E_TO_FIX;
            out[k] = e;
            u += e;
        }
        out[LA_N_TERMS] = u;
        out[LA_N_TERMS + 1] = d.s[w];
    }
    const double *th = d.wth + (size_t)w * 2 * d.P_max;
    for (int p = t; p < P; p += blockDim.x) {
        out[LA_N_TERMS + 2 + p] = th[p];
        out[LA_N_TERMS + 2 + P + p] = th[d.P_max + p];
    }
}

void launch_positions_in(const Dev &d, int w, int n, const float *x, cudaStream_t s) {
    k_positions_in<<<(n + 255) / 256, 256, 0, s>>>(d, w, n, x);
}

void launch_alch_params_in(const Dev &d, int sys, int n_alch, const double *theta, cudaStream_t s) {
    k_alch_params_in<<<1, 256, 0, s>>>(d, sys, theta);
    (void)n_alch;
}

void launch_ef_out(const Dev &d, int w, int P, double *out, cudaStream_t s) {
    k_ef_out<<<1, 128, 0, s>>>(d, w, P, out);
}

void launch_state_io(const Dev &d, int w, int n, float *x, float *v, bool to_slots, cudaStream_t s) {
    k_state_io<<<(n + 255) / 256, 256, 0, s>>>(d, w, n, x, v, to_slots ? 1 : 0);
}

void launch_forces_out(const Dev &d, int w, int n, float *out, cudaStream_t s) {
    k_forces_out<<<(n + 255) / 256, 256, 0, s>>>(d, w, n, out);
}

void launch_lambda_path(const double *lam, int n, double bv, double be, double *out, cudaStream_t s) {
    k_lambda_path<<<(n + 255) / 256, 256, 0, s>>>(lam, n, bv, be, out);
}

}  // namespace labf
