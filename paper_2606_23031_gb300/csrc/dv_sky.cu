// Sky composite (Sec. 3.2 "Sky Modeling", Eq. 2): C = C_voxels + T_final * C_sky(d).
//
// C_sky is a bilinear lookup of an equirectangular environment map of the world
// frame (z up): column coordinate (atan2(d_y, d_x) + pi) / (2 pi) * W, row
// coordinate acos(d_z) / pi * H, texel values at texel centres, wrap-around in
// longitude, clamp to the first / last row in latitude.  One thread per pixel;
// the map (a few MB at most) stays in L2 / L1 while the per-pixel images stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dv_internal.cuh"

namespace dv {

namespace {

struct Tap {
    int idx[4];   // texel offsets (row * W + column) of the four taps
    float w[4];   // their bilinear weights
};

__device__ __forceinline__ Tap sky_taps(const SkyView& v, int u, int px_v, int He, int We) {
    const float xc = ((float)u + 0.5f - v.cx) / v.fx;
    const float yc = ((float)px_v + 0.5f - v.cy) / v.fy;
    float d[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) d[r] = fmaf(v.R[r * 3 + 0], xc, fmaf(v.R[r * 3 + 1], yc, v.R[r * 3 + 2]));
    const float inv = rsqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
    const float lon = atan2f(d[1] * inv, d[0] * inv);
    const float polar = acosf(fminf(fmaxf(d[2] * inv, -1.0f), 1.0f));
    const float x = (lon + 3.14159265358979323846f) * ((float)We * 0.15915494309189535f) - 0.5f;
    const float y = polar * ((float)He * 0.31830988618379067f) - 0.5f;
    const float x0 = floorf(x), y0 = floorf(y);
    const float fx = x - x0, fy = y - y0;
    int i0 = (int)x0 % We;
    if (i0 < 0) i0 += We;
    const int i1 = i0 + 1 == We ? 0 : i0 + 1;
    const int j0 = min(max((int)y0, 0), He - 1), j1 = min(max((int)y0 + 1, 0), He - 1);
    Tap t;
    t.idx[0] = j0 * We + i0;
    t.idx[1] = j0 * We + i1;
    t.idx[2] = j1 * We + i0;
    t.idx[3] = j1 * We + i1;
    t.w[0] = (1.0f - fx) * (1.0f - fy);
    t.w[1] = fx * (1.0f - fy);
    t.w[2] = (1.0f - fx) * fy;
    t.w[3] = fx * fy;
    return t;
}

__global__ void __launch_bounds__(256) k_sky_fwd(const SkyView v, const float* __restrict__ env, int He, int We,
                                                 const float* __restrict__ rgb, const float* __restrict__ alpha,
                                                 float* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)v.W * v.H) return;
    const Tap t = sky_taps(v, (int)(p % v.W), (int)(p / v.W), He, We);
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float* e = env + (size_t)t.idx[k] * 3;
        s0 = fmaf(t.w[k], __ldg(e + 0), s0);
        s1 = fmaf(t.w[k], __ldg(e + 1), s1);
        s2 = fmaf(t.w[k], __ldg(e + 2), s2);
    }
    const float T = 1.0f - alpha[p];
    out[p * 3 + 0] = fmaf(T, s0, rgb[p * 3 + 0]);
    out[p * 3 + 1] = fmaf(T, s1, rgb[p * 3 + 1]);
    out[p * 3 + 2] = fmaf(T, s2, rgb[p * 3 + 2]);
}

// dL/d env += (1 - alpha) w dL/dC at the four taps; dL/d alpha -= dL/dC . C_sky (one pixel
// per thread, so the alpha gradient needs no atomic).  Neighbouring pixels share texels, so the
// lanes of a warp that hit the same texel first sum their parts (match_any + shared memory) and
// one of them adds the sum.
__global__ void __launch_bounds__(256) k_sky_bwd(const SkyView v, const float* __restrict__ env, int He, int We,
                                                 const float* __restrict__ alpha, const float* __restrict__ d_out,
                                                 float* __restrict__ d_env, float* __restrict__ d_alpha) {
    __shared__ float s_part[8][32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = p < (int64_t)v.W * v.H;
    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    if (in) {
        g0 = d_out[p * 3 + 0];
        g1 = d_out[p * 3 + 1];
        g2 = d_out[p * 3 + 2];
    }
    const bool active = in && (g0 != 0.0f || g1 != 0.0f || g2 != 0.0f);
    if (!__any_sync(0xffffffffu, active)) return;  // warp-uniform exit
    Tap t;
    float T = 0.0f;
    if (active) {
        t = sky_taps(v, (int)(p % v.W), (int)(p / v.W), He, We);
        T = 1.0f - alpha[p];
    }
    float dot = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int key = active ? t.idx[k] : -1 - lane;  // inactive lanes never share a key
        if (active) {
            const float* e = env + (size_t)t.idx[k] * 3;
            dot = fmaf(t.w[k], fmaf(g0, __ldg(e + 0), fmaf(g1, __ldg(e + 1), g2 * __ldg(e + 2))), dot);
        }
        if (d_env) {
            const float s = active ? T * t.w[k] : 0.0f;
            s_part[warp][lane][0] = s * g0;
            s_part[warp][lane][1] = s * g1;
            s_part[warp][lane][2] = s * g2;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            __syncwarp();
            if (active && lane == __ffs(peers) - 1) {
                float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
                for (unsigned m = peers; m; m &= m - 1) {
                    const int l = __ffs(m) - 1;
                    a0 += s_part[warp][l][0];
                    a1 += s_part[warp][l][1];
                    a2 += s_part[warp][l][2];
                }
                float* de = d_env + (size_t)t.idx[k] * 3;
                if (a0 != 0.0f) atomicAdd(de + 0, a0);
                if (a1 != 0.0f) atomicAdd(de + 1, a1);
                if (a2 != 0.0f) atomicAdd(de + 2, a2);
            }
            __syncwarp();
        }
    }
    if (active && d_alpha) d_alpha[p] -= dot;
}

}  // namespace

cudaError_t launch_sky_fwd(const SkyView& v, const float* env, int He, int We, const float* rgb, const float* alpha,
                           float* out, cudaStream_t s) {
    const int64_t n = (int64_t)v.W * v.H;
    if (n <= 0) return cudaSuccess;
    k_sky_fwd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, env, He, We, rgb, alpha, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sky_bwd(const SkyView& v, const float* env, int He, int We, const float* alpha, const float* d_out,
                           float* d_env, float* d_alpha, cudaStream_t s) {
    const int64_t n = (int64_t)v.W * v.H;
    if (n <= 0) return cudaSuccess;
    k_sky_bwd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, env, He, We, alpha, d_out, d_env, d_alpha);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dv
