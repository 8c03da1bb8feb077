// Measurement utility: the FP32 FMA issue rate of the device, the denominator of the
// compositing kernels' ALU roofline.  Every thread runs eight independent chains of dependent
// FMAs (enough independent work per warp to cover the FMA latency at full occupancy); the grid
// fills every SM several times over.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dv.h"
#include "dv_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_rate(int iters, float seed, float* __restrict__ out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x * kChains + c) * 1e-7f;
    const float m = 0.99999994f, b = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" dv_status dv_measure_fp32_fma(int32_t device, int32_t iters, int32_t reps, double* flops, double* ms) {
    if (!flops || !ms || iters < 1 || reps < 1) return DV_ERR_INVALID_ARG;
    *flops = 0.0;
    *ms = 0.0;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return DV_ERR_INVALID_ARG;
    const int blocks = dv::sm_count() * 8;  // 8 CTAs of 256 threads per SM: full occupancy
    float* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync(&out, sizeof(float) * (size_t)blocks * kThreads, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fma_rate<<<blocks, kThreads, 0, s>>>(iters, 1.0f, out);  // warm-up (clocks, code load)
        e = cudaEventRecord(e0, s);
    }
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        k_fma_rate<<<blocks, kThreads, 0, s>>>(iters, 1.0f + (float)r, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (out) cudaFreeAsync(out, s);
    if (s) cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return DV_ERR_CUDA;
    dv::count_launches(reps + 1);
    *flops = 2.0 * kChains * kUnroll * (double)iters * (double)blocks * kThreads * (double)reps;
    *ms = t;
    return DV_OK;
}
