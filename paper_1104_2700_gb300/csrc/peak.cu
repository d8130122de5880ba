// Arithmetic-pipe calibration: the FP32 (FFMA) and FP64 (DFMA) throughput of
// the device, measured with independent fused multiply-add chains.  These are
// the denominators against which the force kernels' ALU roofline is checked;
// the paper has no counterpart (its peaks are the CPU's nominal SIMD rates).
#include <cuda_runtime.h>

#include <algorithm>

#include "nbody.h"

namespace {

constexpr int CHAINS = 8;   // independent accumulators per thread (> FMA latency)
constexpr int UNROLL = 8;   // FMAs per chain per loop trip
constexpr int THREADS = 256;
constexpr int BLOCKS_PER_SM = 8;

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Every thread runs CHAINS independent chains x <- x * b + c (b just below 1,
// so the values stay bounded) and writes their sum, so nothing is dead code.
template <typename T>
__global__ void __launch_bounds__(THREADS) fma_throughput_kernel(T* out, T b, T c, int iters)
{
    T x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = static_cast<T>(threadIdx.x + k) * static_cast<T>(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) x[k] = fma_rn(x[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    out[static_cast<size_t>(blockIdx.x) * THREADS + threadIdx.x] = s;
}

// Best of `reps` timed launches (after one warm-up), in TFLOP/s (an FMA = 2 flop).
template <typename T>
cudaError_t time_fma(int sms, int iters, int reps, cudaStream_t st, double* tflops)
{
    const int grid = sms * BLOCKS_PER_SM;
    T* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc(&out, sizeof(T) * static_cast<size_t>(grid) * THREADS);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    double best = 0.0;
    for (int r = 0; r <= reps && err == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        fma_throughput_kernel<T><<<grid, THREADS, 0, st>>>(out, static_cast<T>(0.999999),
                                                           static_cast<T>(1e-6), iters);
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && r > 0 && ms > 0.f) {
            const double flop = 2.0 * CHAINS * UNROLL * static_cast<double>(iters) *
                                static_cast<double>(grid) * THREADS;
            best = std::max(best, flop / (ms * 1e-3) / 1e12);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    *tflops = best;
    return err;
}

}  // namespace

extern "C" nb_status nb_measure_peaks(int32_t device, double* fp32_tflops, double* fp64_tflops)
{
    if (!fp32_tflops || !fp64_tflops) return NB_EINVAL;
    *fp32_tflops = 0.0;
    *fp64_tflops = 0.0;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return NB_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return NB_EINVAL;
    int sms = 0;
    cudaStream_t st = nullptr;
    cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    // ~20 ms per FP32 launch at ~80 TFLOP/s; the FP64 pipe is far narrower on
    // this part, so its chains are 1/64 as long.
    if (err == cudaSuccess) err = time_fma<float>(sms, 40000, 3, st, fp32_tflops);
    if (err == cudaSuccess) err = time_fma<double>(sms, 625, 3, st, fp64_tflops);
    if (st) cudaStreamDestroy(st);
    cudaSetDevice(prev);
    return err == cudaSuccess ? NB_OK : NB_ECUDA;
}
