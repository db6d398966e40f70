// Arithmetic peak of this GPU, measured: independent fused multiply-add
// chains in every thread of a full grid, timed with CUDA events.  The
// roofline of the FP64 operator apply (bound by FP64 arithmetic on GB300)
// is quoted against this number instead of a nominal figure.
#include <cuda_runtime.h>

#include "ht.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(int iters, T b, T c, T* __restrict__ sink) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == (T)-1.2345) sink[0] = s;   // never true; keeps the chains live
}

template <typename T>
int run_probe(int device, int iters, int reps, double* tflops) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return HT_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    T* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HT_OK;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = HT_ECUDA;
    const int blocks = sms * 8, threads = 256;
    double best = 0.0;
    for (int r = 0; r <= reps && rc == HT_OK; ++r) {   // r = 0 is a warm-up launch
        cudaEventRecord(e0);
        fma_chains_kernel<T><<<blocks, threads>>>(iters, (T)0.999999, (T)1e-7, sink);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) { rc = HT_ECUDA; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * kChains * (double)iters * blocks * threads;
        if (r > 0 && ms > 0.0f && flops / (ms * 1e-3) / 1e12 > best) best = flops / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (prev >= 0) cudaSetDevice(prev);
    *tflops = best;
    return rc;
}

}  // namespace

extern "C" int ht_fma_peak(int device, int fp64, double* tflops) {
    if (!tflops) return HT_EINVAL;
    *tflops = 0.0;
    return fp64 ? run_probe<double>(device, 1 << 12, 5, tflops) : run_probe<float>(device, 1 << 16, 5, tflops);
}
