// k_io.cu -- state and force transfer between the slot layout and the
// system's atom order, and the lambda-path evaluator.
#include "labf_internal.cuh"
#include "labf_launch.h"

namespace labf {

// to_slots = 0: x, v (atom order) <- slots;  1: slots <- x, v
__global__ void k_state_io(Dev d, int w, int n, float *x, float *v, int to_slots) {
    const WalkerDev &W = d.walk[w];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = d.slot_of_atom[W.atom_base + i];
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
        const int g = d.slot_of_atom[W.atom_base + i];
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
