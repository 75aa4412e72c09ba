// Measured FMA throughput of the device in FP64 and FP32: the ALU roof of the kernels that are bound by arithmetic
// rather than by memory (the FP64 outer residual).  The paper reports no such figure; this is a measurement helper of
// the library, used by its benchmark to report those kernels against a measured rather than a derived peak.
#include <cuda_runtime.h>

#include <string>

#include "octmg_internal.h"

namespace octmg {
namespace {

// Eight independent FMA chains per thread (enough to fill the pipes), values kept bounded (a -> c / (1 - b)); the
// result is written only if it takes an impossible value, so the chains stay live without memory traffic.
template <typename T>
__global__ void k_fma_rate(T *out, int iters, T b, T c) {
    T a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = T(threadIdx.x + q) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = fma(a[q], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) s += a[q];
    if (s == T(-1)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// TFLOP/s (2 flop per FMA) of one timed launch after a warm-up one; 0 on a CUDA error.
template <typename T>
double fma_tflops(int sms, int iters) {
    const int threads = 256, blocks = sms * 8;
    T *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double r = 0.0;
    if (cudaMalloc(&out, sizeof(T) * threads * blocks) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        k_fma_rate<T><<<blocks, threads>>>(out, iters / 4, T(0.999999), T(1e-6));
        cudaEventRecord(e0);
        k_fma_rate<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-6));
        cudaEventRecord(e1);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f)
            r = 2.0 * 8.0 * static_cast<double>(iters) * threads * blocks / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return r;
}

}  // namespace
}  // namespace octmg

extern "C" mg_status mg_alu_peaks(double *fp64_tflops, double *fp32_tflops) {
    if (!fp64_tflops && !fp32_tflops) {
        octmg::set_error("mg_alu_peaks: no output");
        return MG_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        octmg::set_error("mg_alu_peaks: no CUDA device");
        return MG_ERR_CUDA;
    }
    if (fp64_tflops && (*fp64_tflops = octmg::fma_tflops<double>(sms, 4000)) <= 0.0) {
        octmg::set_error("mg_alu_peaks: the FP64 probe failed");
        return MG_ERR_CUDA;
    }
    if (fp32_tflops && (*fp32_tflops = octmg::fma_tflops<float>(sms, 100000)) <= 0.0) {
        octmg::set_error("mg_alu_peaks: the FP32 probe failed");
        return MG_ERR_CUDA;
    }
    return MG_OK;
}
