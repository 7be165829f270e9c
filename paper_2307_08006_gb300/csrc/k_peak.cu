// k_peak.cu -- measured arithmetic peaks for the roofline of the pair pass:
// FP32 fused multiply-adds (the CUDA-core rate the pair kernel is bound by)
// and FP64 fused multiply-adds (the rate of the few FP64 paths), each timed
// with CUDA events over a stream of independent FMA chains on every SM.
#include <cuda_runtime.h>

#include "labf.h"

namespace labf {
namespace {

constexpr int CHAINS = 8;  // independent FMA chains per thread (covers the pipe latency)

__device__ double g_peak_sink[256];  // written only if a chain ends at -1 (never): keeps the chains live

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T b, T c) {
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == (T)-1) g_peak_sink[threadIdx.x] = (double)s;
}

template <typename T>
int time_fma(int n_sm, double seconds, cudaStream_t s, double *tflops) {
    const int blocks = n_sm * 8, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LA_ERR_CUDA;
    int iters = sizeof(T) == 4 ? 4096 : 64;
    float ms = 0.f;
    int rc = LA_OK;
    // warm up, then grow the launch until it lasts about `seconds`
    for (int pass = 0; pass < 8; ++pass) {
        cudaEventRecord(e0, s);
        k_fma_peak<T><<<blocks, threads, 0, s>>>(iters, (T)0.9999, (T)1e-4);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = LA_ERR_CUDA;
            break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        if (pass > 0 && ms >= 0.5e3 * seconds) break;
        const double grow = ms > 0.f ? 1e3 * seconds / ms : 16.0;
        const double next = (double)iters * (grow < 16.0 ? (grow > 1.0 ? grow : 1.0) : 16.0);
        iters = next > 2e9 ? 2000000000 : (int)next;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LA_OK || ms <= 0.f) return LA_ERR_CUDA;
    const double flops = 2.0 * CHAINS * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return LA_OK;
}

}  // namespace
}  // namespace labf

extern "C" int la_fp_peak(int fp64, double seconds, double *tflops, void *stream) {
    if (!tflops || !(seconds > 0.0) || seconds > 10.0) return LA_ERR_INVALID_ARG;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LA_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    return fp64 ? labf::time_fma<double>(n_sm, seconds, s, tflops) : labf::time_fma<float>(n_sm, seconds, s, tflops);
}
