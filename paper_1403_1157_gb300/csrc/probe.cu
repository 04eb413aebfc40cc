// cdg2_probe_peak: the FMA throughput of this GPU in FP64 or FP32, measured
// with an FMA loop, so that the roofline fractions of the operator kernels
// (bound by the FP64 or FP32 pipes, not by HBM) are stated against a measured
// peak.  The paper has no counterpart; this is a measurement utility.
#include "cdg2_internal.h"

namespace cdg2 {

static __device__ double g_probe_sink;

// Every thread runs CH independent FMA chains of `iters` steps (enough chains
// to hide the pipe latency); the values depend on the thread so nothing folds,
// and a store the compiler cannot rule out keeps the loop alive (the chains
// grow monotonically from 0, so their sum is never negative).
template <typename T, int CH>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters) {
    T a[CH];
    const T x = T(1) + T(threadIdx.x) * T(1e-7);
    const T y = T(1) - T(blockIdx.x) * T(1e-9);
#pragma unroll
    for (int c = 0; c < CH; ++c) a[c] = T(c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) a[c] = fma(a[c], x, y);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CH; ++c) s += a[c];
    if (s < T(0)) g_probe_sink = double(s);
}

template <typename T>
static int run_probe(int iters, double* tflops, cudaStream_t st) {
    constexpr int CH = 8;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_probe_peak");
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t a, b;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_probe_peak");
    fma_probe_kernel<T, CH><<<blocks, threads, 0, st>>>(iters / 8);   // warm-up
    cudaEventRecord(a, st);
    fma_probe_kernel<T, CH><<<blocks, threads, 0, st>>>(iters);
    cudaEventRecord(b, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_probe_peak");
    const double flops = 2.0 * CH * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return CDG2_OK;
}

}  // namespace cdg2

using namespace cdg2;

extern "C" int cdg2_probe_peak(int kind, int iters, double* tflops, void* stream) {
    if (!tflops || iters < 8 || (kind != 0 && kind != 1)) {
        set_error("cdg2_probe_peak: kind must be 0 (FP64) or 1 (FP32), iters >= 8, tflops non-NULL");
        return CDG2_ERR_INVALID_ARG;
    }
    return kind == 0 ? run_probe<double>(iters, tflops, (cudaStream_t)stream)
                     : run_probe<float>(iters, tflops, (cudaStream_t)stream);
}
