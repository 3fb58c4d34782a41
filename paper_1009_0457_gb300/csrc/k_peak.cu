// Peak FP32 and FP64 fused multiply-add rate of the device, measured: the denominator
// beside the derived peak (SMs x lanes x 2 x clock) for the ALU-bound kernels.  Every
// thread runs eight independent multiply-add chains (so the pipes never wait on a
// dependency) over a grid of several resident CTAs per SM; the chains' values are kept
// alive by a store that the data never triggers.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hmc.h"

namespace {

constexpr int PEAK_THREADS = 256, PEAK_CHAINS = 8, PEAK_UNROLL = 16;
// bounds one launch to a few seconds at GB300's FP64 rate
constexpr int PEAK_MAX_ITERS = 1 << 16;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(T *sink, int iters, T m, T c) {
    T a[PEAK_CHAINS];
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = T(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
            for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = fma(a[j], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) s += a[j];
    if (s == T(-1.0e30)) sink[blockIdx.x] = s;   // never true: keeps the chains
}

template <typename T>
cudaError_t measure(int iters, double *tflops) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, PEAK_THREADS, 0)) != cudaSuccess)
        return e;
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    T *sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(T) * (size_t)grid)) != cudaSuccess) return e;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const T m = T(0.9999999), c = T(1.0e-7);
    // one warm-up launch, then the best of three
    if (e == cudaSuccess) {
        k_fma_peak<T><<<grid, PEAK_THREADS, 0, s>>>(sink, iters, m, c);
        e = cudaGetLastError();
    }
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        float ms = 0.f;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        k_fma_peak<T><<<grid, PEAK_THREADS, 0, s>>>(sink, iters, m, c);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        if (ms < best) best = ms;
    }
    if (e == cudaSuccess) {
        const double flop = 2.0 * PEAK_CHAINS * PEAK_UNROLL * (double)iters * PEAK_THREADS * grid;
        *tflops = flop / (best * 1e-3) / 1e12;
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    return e;
}

}  // namespace

extern "C" hmc_status hmc_fma_peak(int32_t precision, int32_t iters, double *tflops) {
    if (!tflops || iters < 1 || iters > PEAK_MAX_ITERS || (precision != HMC_FP32 && precision != HMC_FP64)) return HMC_ERR_ARG;
    const cudaError_t e = precision == HMC_FP32 ? measure<float>(iters, tflops) : measure<double>(iters, tflops);
    return e == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}
