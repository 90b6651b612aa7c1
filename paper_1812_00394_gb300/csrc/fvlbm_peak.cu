// FP64 arithmetic peak of the device, measured: the FP64 path of the step is bound by the FP64
// pipe (not by memory), and its roofline is the rate of fused multiply-adds this GPU sustains.
// Each thread runs kChains independent FMA chains for `iters` iterations; nothing is read from
// memory, and the results are summed into one store per thread so that no chain is dead code.
#include <cuda_runtime.h>

#include "fvlbm.h"

namespace {

constexpr int kChains = 8;

__global__ void k_fp64_fma(int iters, double a, double b, double *__restrict__ out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = a + c * 1e-3 + threadIdx.x * 1e-9;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], b, a);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int fvlbm_fp64_peak(int device, double *tflops) {
    if (!tflops) return FVLBM_ERR_BAD_PARAM;
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return FVLBM_ERR_CUDA;
    if (cudaSetDevice(dev) != cudaSuccess) return FVLBM_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FVLBM_ERR_CUDA;
    const int threads = 256, blocks = sms * 8, iters = 4096;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * static_cast<size_t>(threads) * blocks) != cudaSuccess)
        return FVLBM_ERR_OOM;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, s);
        k_fp64_fma<<<blocks, threads, 0, s>>>(iters, 0.5, 0.999999, out);
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    if (err != cudaSuccess) return FVLBM_ERR_CUDA;
    const double flops = 2.0 * kChains * static_cast<double>(iters) * threads * blocks;
    *tflops = flops / (static_cast<double>(best) * 1e-3) / 1e12;
    return FVLBM_OK;
}
