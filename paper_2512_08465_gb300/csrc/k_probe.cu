// ALU peak probe for the roofline of the FP64 path: many independent fused
// multiply-add chains per thread, enough resident warps per SM to fill the
// pipes, timed with CUDA events.  Reported as FLOP/s (2 per FMA).
#include <cstdio>

#include "cs_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;

template <typename T>
__global__ void fma_probe(T* out, T a, T b) {
    T x[kChains];
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)123.456) out[blockIdx.x] = s;      // keeps the chains live
}

template <typename T>
double probe(int sms, T* buf) {
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_probe<T><<<blocks, threads>>>(buf, (T)0.999999, (T)1e-7);
    cudaEventRecord(e0);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) fma_probe<T><<<blocks, threads>>>(buf, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * kChains * kIters * (double)blocks * threads * reps;
    return flops / (ms * 1e-3) / 1e12;
}

}  // namespace

extern "C" cs_status cs_alu_peak(int32_t device, double* fp64_tflops, double* fp32_tflops) {
    if (!fp64_tflops || !fp32_tflops) return CS_E_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return CS_E_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return CS_E_CUDA;
    void* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * sms * 8) != cudaSuccess) return CS_E_NOMEM;
    *fp64_tflops = probe<double>(sms, (double*)buf);
    *fp32_tflops = probe<float>(sms, (float*)buf);
    cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    return e == cudaSuccess ? CS_OK : CS_E_CUDA;
}
