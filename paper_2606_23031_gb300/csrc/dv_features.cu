// Feature fields over the compositing weights (Sec. 4, "3D Semantic Segmentation" and "Open
// Vocabulary Scene Understanding": the renderer's RGB accumulation with the colour replaced by a
// high-dimensional per-voxel feature, and the fusion of 2-D features into the voxels).
//
// A render's weights export lists, for every pixel p, the composited segments' voxel indices
// and weights w = T alpha in slots [off[p], off[p+1]).  Then
//   render:  F[p][c]  = sum_slots w * feat[voxel][c]
//   fuse:    acc[v][c] += sum over the slots of voxel v of w * F2d[p][c],  wsum[v] += w
// One warp per pixel, one lane per channel (32 channels per pass over the slots), so each
// feature row is read with coalesced loads.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dv_internal.cuh"

namespace dv {

namespace {

constexpr int FT_WARPS = 8;  // pixels per 256-thread block

__global__ void __launch_bounds__(FT_WARPS * 32) k_feat_render(int64_t n_pix, const int64_t* __restrict__ off,
                                                               const uint32_t* __restrict__ vox,
                                                               const float* __restrict__ wgt,
                                                               const float* __restrict__ feat, int C,
                                                               float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * FT_WARPS + (threadIdx.x >> 5);
    if (p >= n_pix) return;
    const int64_t e0 = off[p], e1 = off[p + 1];
    for (int c0 = 0; c0 < C; c0 += 32) {
        const int c = c0 + lane;
        float acc = 0.0f;
        for (int64_t e = e0; e < e1; ++e) {
            const float w = __ldg(wgt + e);
            const uint32_t v = __ldg(vox + e);
            if (c < C) acc = fmaf(w, __ldg(feat + (size_t)v * C + c), acc);
        }
        if (c < C) out[(size_t)p * C + c] = acc;
    }
}

__global__ void __launch_bounds__(FT_WARPS * 32) k_feat_fuse(int64_t n_pix, const int64_t* __restrict__ off,
                                                             const uint32_t* __restrict__ vox,
                                                             const float* __restrict__ wgt,
                                                             const float* __restrict__ f2d, int C,
                                                             float* __restrict__ acc, float* __restrict__ wsum) {
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * FT_WARPS + (threadIdx.x >> 5);
    if (p >= n_pix) return;
    const int64_t e0 = off[p], e1 = off[p + 1];
    for (int64_t e = e0; e < e1; ++e) {
        const float w = __ldg(wgt + e);
        if (w == 0.0f) continue;
        const uint32_t v = __ldg(vox + e);
        for (int c = lane; c < C; c += 32) atomicAdd(acc + (size_t)v * C + c, w * __ldg(f2d + (size_t)p * C + c));
        if (wsum && lane == 0) atomicAdd(wsum + v, w);
    }
}

}  // namespace

cudaError_t launch_feat_render(int64_t n_pix, const int64_t* off, const uint32_t* vox, const float* wgt,
                               const float* feat, int C, float* out, cudaStream_t s) {
    if (n_pix <= 0 || C <= 0) return cudaSuccess;
    k_feat_render<<<(unsigned)((n_pix + FT_WARPS - 1) / FT_WARPS), FT_WARPS * 32, 0, s>>>(n_pix, off, vox, wgt, feat,
                                                                                           C, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_feat_fuse(int64_t n_pix, const int64_t* off, const uint32_t* vox, const float* wgt,
                             const float* f2d, int C, float* acc, float* wsum, cudaStream_t s) {
    if (n_pix <= 0 || C <= 0) return cudaSuccess;
    k_feat_fuse<<<(unsigned)((n_pix + FT_WARPS - 1) / FT_WARPS), FT_WARPS * 32, 0, s>>>(n_pix, off, vox, wgt, f2d, C,
                                                                                         acc, wsum);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dv
