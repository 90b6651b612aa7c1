// fvlbm_noalloc.cu -- an entry point for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while another component owns every
// allocation (a framework's caching allocator, a memory pool sized once at start-up), real-time
// loops that must not block on the allocator, or embedded drivers that forbid allocation after
// initialisation.  fvlbm_stats_reduce_static gives them the FP64 residual / mass / NaN reduction
// of a time step without any allocation: its per-block partial sums live in a fixed file-scope
// device array instead of a buffer from cudaMalloc.  The paper has no counterpart; this is a
// deployment convenience around the reduction the time step already performs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "fvlbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = FVLBM_STATS_STATIC_MAX_CELLS / kThreads;  // 16384 blocks
constexpr int kMaxDevices = 64;

// Scratch for the per-block partial sums: kMaxBlocks x 4 doubles = 512 KiB on every device that
// loads the library, held until the process exits.  Every call overwrites exactly the partials
// it reads back, so nothing has to be cleared between calls.  Calls that overlap on the GPU
// (two streams, or two host threads) share this array and race.
__device__ __align__(256) double g_partials[kMaxBlocks * 4];

std::mutex g_mu;
double *g_partials_addr[kMaxDevices] = {nullptr};

// Device address of g_partials on the current device (the host-side symbol is only a
// stand-in and must never be passed to a kernel).  The first call on a device looks it up.
// Later calls look it up again whenever `stream` is not being captured, so that a context
// that was reset (cudaDeviceReset) and loaded the module anew is never handed a stale
// address; while a capture is under way the address cached by the last lookup is used, since
// a lookup might load the module and that is not allowed during a capture.
cudaError_t partials_address(int device, cudaStream_t stream, double **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusActive;
    if (!g_partials_addr[device] || cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[device] = static_cast<double *>(p);
    }
    *out = g_partials_addr[device];
    return cudaSuccess;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per block: sum |u_new - u_old|^2, sum |u_new|^2, sum rho A and the count of non-finite cells.
__global__ void __launch_bounds__(kThreads)
    k_stats_partials(const double *__restrict__ u_old, const double *__restrict__ v_old,
                     const double *__restrict__ u_new, const double *__restrict__ v_new,
                     const double *__restrict__ rho, const double *__restrict__ area, int n,
                     double *__restrict__ partials) {
    __shared__ double red[kThreads / 32][4];
    const int i = blockIdx.x * kThreads + threadIdx.x;
    double s[4] = {0, 0, 0, 0};
    if (i < n) {
        const double du = u_new[i] - u_old[i], dv = v_new[i] - v_old[i];
        s[0] = du * du + dv * dv;
        s[1] = u_new[i] * u_new[i] + v_new[i] * v_new[i];
        s[2] = rho[i] * area[i];
        s[3] = (isfinite(u_new[i]) && isfinite(v_new[i]) && isfinite(rho[i])) ? 0.0 : 1.0;
    }
    for (int k = 0; k < 4; ++k) s[k] = warp_sum(s[k]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) red[warp][k] = s[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w][threadIdx.x];
        partials[4 * blockIdx.x + threadIdx.x] = t;
    }
}

// One block folds the partials: out = {sum du^2, sum u^2, mass, non-finite count}.
__global__ void __launch_bounds__(kThreads)
    k_stats_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
    __shared__ double red[kThreads / 32][4];
    double s[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int k = 0; k < 4; ++k) s[k] += partials[4 * b + k];
    for (int k = 0; k < 4; ++k) s[k] = warp_sum(s[k]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) red[warp][k] = s[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

}  // namespace

extern "C" int fvlbm_stats_reduce_static(const double *u_old, const double *v_old,
                                         const double *u_new, const double *v_new,
                                         const double *rho, const double *area, int n,
                                         double *out, void *stream) {
    if (n < 0 || !out || (n > 0 && (!u_old || !v_old || !u_new || !v_new || !rho || !area)))
        return FVLBM_ERR_BAD_PARAM;
    if (n > FVLBM_STATS_STATIC_MAX_CELLS) {
        fprintf(stderr,
                "fvlbm_stats_reduce_static: %d cells exceed the static scratch capacity of %d "
                "cells\n",
                n, FVLBM_STATS_STATIC_MAX_CELLS);
        return FVLBM_ERR_BAD_PARAM;
    }
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
        return FVLBM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *partials = nullptr;
    if (partials_address(device, s, &partials) != cudaSuccess) return FVLBM_ERR_CUDA;
    const int nblocks = (n + kThreads - 1) / kThreads;
    if (nblocks > 0)
        k_stats_partials<<<nblocks, kThreads, 0, s>>>(u_old, v_old, u_new, v_new, rho, area, n,
                                                      partials);
    k_stats_final<<<1, kThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError() == cudaSuccess ? FVLBM_OK : FVLBM_ERR_CUDA;
}
