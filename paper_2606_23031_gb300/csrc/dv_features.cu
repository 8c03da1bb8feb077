// Feature fields over the compositing weights (Sec. 4, "3D Semantic Segmentation" and "Open
// Vocabulary Scene Understanding": the renderer's RGB accumulation with the colour replaced by a
// high-dimensional per-voxel feature, and the fusion of 2-D features into the voxels).
//
// A render's weights export lists, for every pixel p, the composited segments' voxel indices
// and weights w = T alpha in slots [off[p], off[p+1]).  Then
//   render:  F[p][c]  = sum_slots w * feat[voxel][c]
//   fuse:    acc[v][c] += sum over the slots of voxel v of w * F2d[p][c],  wsum[v] += w
// Render: one warp per pixel.  When C is a multiple of 4 whose quads divide the warp (C = 4, 8,
// ..., 64, 128) a lane owns a 16-byte quad of channels and the warp covers 32 / (C / 4) slots at
// once; other C take one lane per channel, 32 channels per pass over the slots.
// Fusion: adding every slot into its voxel's row with its own atomics is bound by the L2's
// atomic rate (one add per slot and channel), so the slots are first sorted by voxel and each
// run of one voxel is summed in registers and added once.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dv_internal.cuh"

namespace dv {

namespace {

constexpr int FT_WARPS = 8;  // pixels per 256-thread block

// Scalar path (any C): one lane per channel, 32 channels per pass over the slots.
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

// Vector path (C = 4 Q with Q dividing 32): a lane owns one 16-byte quad of channels and the warp
// walks S = 32 / Q slots at a time, lane group g taking slots e0 + g, e0 + g + S, ...; the S
// partial sums of a quad are then added across the groups with shuffles.
__global__ void __launch_bounds__(FT_WARPS * 32) k_feat_render4(int64_t n_pix, const int64_t* __restrict__ off,
                                                                const uint32_t* __restrict__ vox,
                                                                const float* __restrict__ wgt,
                                                                const float4* __restrict__ feat, int Q,
                                                                float4* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * FT_WARPS + (threadIdx.x >> 5);
    if (p >= n_pix) return;
    const int S = 32 / Q, q = lane % Q, g = lane / Q;
    const int64_t e0 = off[p], e1 = off[p + 1];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t e = e0 + g; e < e1; e += S) {
        const float w = __ldg(wgt + e);
        const float4 f = __ldg(feat + (size_t)__ldg(vox + e) * Q + q);
        acc.x = fmaf(w, f.x, acc.x);
        acc.y = fmaf(w, f.y, acc.y);
        acc.z = fmaf(w, f.z, acc.z);
        acc.w = fmaf(w, f.w, acc.w);
    }
    for (int d = Q; d < 32; d <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, d);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, d);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, d);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, d);
    }
    if (g == 0) out[(size_t)p * Q + q] = acc;
}

// ---- fusion by voxel runs ----
// The slots are sorted by voxel (stable, so a voxel's slots keep their export order); a warp
// takes FZ_CHUNK consecutive sorted slots, sums w * F2d[p] over each run of one voxel in
// registers and adds a run's sums into the voxel's row once.  Atomics drop from one per slot
// and channel to one per run and channel (a run is cut only at chunk ends), and within a run the
// sum is taken in export order.

constexpr int FZ_CHUNK = 256;  // sorted slots per warp

// key = voxel, value = slot, pw[slot] = (pixel, weight bits); the largest voxel index goes to *vmax.
// A block takes FZ_PREP consecutive pixels, whose slots are one contiguous range, and strides over
// that range with coalesced loads and stores; a slot's pixel is the last of the block's offsets at
// or below it (binary search in shared memory).
constexpr int FZ_PREP = 256;
__global__ void __launch_bounds__(FZ_PREP) k_fuse_prep(int64_t n_pix, const int64_t* __restrict__ off,
                                                       const uint32_t* __restrict__ vox, const float* __restrict__ wgt,
                                                       uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                                                       uint2* __restrict__ pw, uint32_t* __restrict__ vmax) {
    __shared__ int64_t s_off[FZ_PREP + 1];
    const int64_t p0 = (int64_t)blockIdx.x * FZ_PREP;
    const int np = (int)min((int64_t)FZ_PREP, n_pix - p0);
    for (int i = threadIdx.x; i <= np; i += FZ_PREP) s_off[i] = off[p0 + i];
    __syncthreads();
    uint32_t m = 0;
    const int64_t e1 = s_off[np];
    for (int64_t e = s_off[0] + threadIdx.x; e < e1; e += FZ_PREP) {
        int lo = 0, hi = np - 1;  // the owner i has s_off[i] <= e < s_off[i + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= e)
                lo = mid;
            else
                hi = mid - 1;
        }
        const uint32_t v = __ldg(vox + e);
        key[e] = v;
        val[e] = (uint32_t)e;
        pw[e] = make_uint2((uint32_t)(p0 + lo), __float_as_uint(__ldg(wgt + e)));
        m = max(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(vmax, m);
}

// Any C: lane owns channels c0 + lane + 32 j, j < CPL; the warp walks its slots in groups of
// FZ_LOOK, issuing their loads together before summing them in order.
constexpr int FZ_LOOK = 4;
template <int CPL>
__global__ void __launch_bounds__(256) k_fuse_runs(int64_t n, const uint32_t* __restrict__ skey,
                                                   const uint32_t* __restrict__ sval, const uint2* __restrict__ pw,
                                                   const float* __restrict__ f2d, int C, float* __restrict__ acc,
                                                   float* __restrict__ wsum) {
    const int lane = threadIdx.x & 31;
    const int64_t i0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * FZ_CHUNK;
    if (i0 >= n) return;
    const int64_t i1 = min(n, i0 + FZ_CHUNK);
    for (int c0 = 0; c0 < C; c0 += 32 * CPL) {
        float a[CPL];
#pragma unroll
        for (int j = 0; j < CPL; ++j) a[j] = 0.0f;
        float ws = 0.0f;
        uint32_t cur = __ldg(skey + i0);
        auto flush = [&]() {
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                const int c = c0 + lane + 32 * j;
                if (c < C && a[j] != 0.0f) atomicAdd(acc + (size_t)cur * C + c, a[j]);
                a[j] = 0.0f;
            }
            if (c0 == 0 && wsum && lane == 0 && ws != 0.0f) atomicAdd(wsum + cur, ws);
            ws = 0.0f;
        };
        for (int64_t i = i0; i < i1; i += FZ_LOOK) {
            uint32_t v[FZ_LOOK];
            float w[FZ_LOOK], f[FZ_LOOK][CPL];
#pragma unroll
            for (int k = 0; k < FZ_LOOK; ++k) {
                const bool in = i + k < i1;
                v[k] = in ? __ldg(skey + i + k) : cur;
                const uint2 q = in ? __ldg(pw + __ldg(sval + i + k)) : make_uint2(0u, 0u);
                w[k] = __uint_as_float(q.y);
                const size_t row = (size_t)q.x * C;
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    const int c = c0 + lane + 32 * j;
                    f[k][j] = (in && c < C) ? __ldg(f2d + row + c) : 0.0f;
                }
            }
#pragma unroll
            for (int k = 0; k < FZ_LOOK; ++k) {
                if (i + k < i1) {
                    if (v[k] != cur) {
                        flush();
                        cur = v[k];
                    }
#pragma unroll
                    for (int j = 0; j < CPL; ++j) a[j] = fmaf(w[k], f[k][j], a[j]);
                    ws += w[k];
                }
            }
        }
        flush();
    }
}

// C = 4 Q with Q | 32: lane (g = lane / Q, q = lane % Q) owns the 16-byte quad q of every
// S-th slot (S = 32 / Q slots per load instruction).  Per 32 sorted slots the warp loads their
// (voxel, slot) and (pixel, weight) with one load each, lane k holding slot k, then R * S slots
// at a time gathers their rows (R loads in flight per lane) and sums them in slot order into
// the running voxel's quads; at a run's end the S partial quads are added across the groups and
// the run is added once.
// (4 rows in flight and 5 resident blocks per SM measured best: 8 rows held 3 blocks, more blocks spilled)
template <int Q, int R = (Q < 4 ? Q : 4)>
__global__ void __launch_bounds__(256, 5) k_fuse_runs4(int64_t n, const uint32_t* __restrict__ skey,
                                                    const uint32_t* __restrict__ sval, const uint2* __restrict__ pw,
                                                    const float4* __restrict__ f2d, float4* __restrict__ acc,
                                                    float* __restrict__ wsum) {
    constexpr int S = 32 / Q;
    const int lane = threadIdx.x & 31, g = lane / Q, q = lane % Q;
    const int64_t i0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * FZ_CHUNK;
    if (i0 >= n) return;
    const int64_t i1 = min(n, i0 + FZ_CHUNK);
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    float ws = 0.0f;
    uint32_t cur = __ldg(skey + i0);
    auto flush = [&]() {
#pragma unroll
        for (int d = Q; d < 32; d <<= 1) {
            a.x += __shfl_xor_sync(0xffffffffu, a.x, d);
            a.y += __shfl_xor_sync(0xffffffffu, a.y, d);
            a.z += __shfl_xor_sync(0xffffffffu, a.z, d);
            a.w += __shfl_xor_sync(0xffffffffu, a.w, d);
        }
        if (g == 0 && (a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f)) atomicAdd(acc + (size_t)cur * Q + q, a);
        if (wsum && lane == 0 && ws != 0.0f) atomicAdd(wsum + cur, ws);
        a = make_float4(0.f, 0.f, 0.f, 0.f);
        ws = 0.0f;
    };
    for (int64_t i = i0; i < i1; i += 32) {
        const int cnt = (int)min((int64_t)32, i1 - i);
        const bool in = lane < cnt;
        const uint32_t v_l = in ? __ldg(skey + i + lane) : 0u;
        const uint2 pw_l = in ? __ldg(pw + __ldg(sval + i + lane)) : make_uint2(0u, 0u);
        const float w_l = __uint_as_float(pw_l.y);
        for (int k0 = 0; k0 < cnt; k0 += S * R) {
            float4 f[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int sl = k0 + r * S + g;  // < 32 + S * R <= 64
                const uint32_t pp = __shfl_sync(0xffffffffu, pw_l.x, sl & 31);
                f[r] = sl < cnt ? __ldg(f2d + (size_t)pp * Q + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll
                for (int h = 0; h < S; ++h) {
                    const int sl = k0 + r * S + h;
                    if (sl < cnt) {  // warp-uniform
                        const uint32_t vv = __shfl_sync(0xffffffffu, v_l, sl);
                        const float ww = __shfl_sync(0xffffffffu, w_l, sl);
                        if (vv != cur) {
                            flush();
                            cur = vv;
                        }
                        if (g == h) {
                            a.x = fmaf(ww, f[r].x, a.x);
                            a.y = fmaf(ww, f[r].y, a.y);
                            a.z = fmaf(ww, f[r].z, a.z);
                            a.w = fmaf(ww, f[r].w, a.w);
                        }
                        ws += ww;
                    }
                }
            }
        }
    }
    flush();
}

// the 16-byte render path needs C = 4 Q with Q a divisor of 32 and 16-byte aligned rows
bool quad_path(int C, const void* a, const void* b) {
    if (C % 4 != 0 || C / 4 > 32 || 32 % (C / 4) != 0) return false;
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

}  // namespace

cudaError_t launch_feat_render(int64_t n_pix, const int64_t* off, const uint32_t* vox, const float* wgt,
                               const float* feat, int C, float* out, cudaStream_t s) {
    if (n_pix <= 0 || C <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n_pix + FT_WARPS - 1) / FT_WARPS);
    if (quad_path(C, feat, out))
        k_feat_render4<<<grid, FT_WARPS * 32, 0, s>>>(n_pix, off, vox, wgt, reinterpret_cast<const float4*>(feat),
                                                      C / 4, reinterpret_cast<float4*>(out));
    else
        k_feat_render<<<grid, FT_WARPS * 32, 0, s>>>(n_pix, off, vox, wgt, feat, C, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t feat_fuse(int64_t n_pix, const int64_t* off, const uint32_t* vox, const float* wgt, const float* f2d,
                      int C, float* acc, float* wsum, Arena& ar, cudaStream_t s, bool* sort_timeout) {
    *sort_timeout = false;
    if (n_pix <= 0 || C <= 0) return cudaSuccess;
    int64_t n = 0;
    cudaError_t e = cudaMemcpyAsync(&n, off + n_pix, sizeof(n), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    if (n > (int64_t)UINT32_MAX || n_pix > (int64_t)UINT32_MAX) return cudaErrorInvalidValue;  // 32-bit slot and pixel indices
    uint32_t* k0 = ar.alloc<uint32_t>(n);
    uint32_t* k1 = ar.alloc<uint32_t>(n);
    uint32_t* v0 = ar.alloc<uint32_t>(n);
    uint32_t* v1 = ar.alloc<uint32_t>(n);
    uint2* pw = ar.alloc<uint2>(n);
    uint32_t* vmax = ar.alloc<uint32_t>(2);  // [0] largest voxel index, [1] the sort's wait flag
    if (ar.err != cudaSuccess) return ar.err;
    e = cudaMemsetAsync(vmax, 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_fuse_prep<<<(unsigned)((n_pix + FZ_PREP - 1) / FZ_PREP), FZ_PREP, 0, s>>>(n_pix, off, vox, wgt, k0, v0, pw, vmax);
    count_launches(1);
    uint32_t vm = 0;
    e = cudaMemcpyAsync(&vm, vmax, sizeof(vm), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    int bits = 0;
    while (bits < 32 && (vm >> bits)) ++bits;
    uint32_t* kk = k0;
    uint32_t* vv = v0;
    e = radix_sort_u32(kk, vv, k1, v1, n, bits, ar, s, vmax + 1);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((n + FZ_CHUNK * 8 - 1) / (FZ_CHUNK * 8));
    const float4* f4 = reinterpret_cast<const float4*>(f2d);
    float4* a4 = reinterpret_cast<float4*>(acc);
    if (quad_path(C, f2d, acc)) {
        switch (C / 4) {
            case 1: k_fuse_runs4<1><<<grid, 256, 0, s>>>(n, kk, vv, pw, f4, a4, wsum); break;
            case 2: k_fuse_runs4<2><<<grid, 256, 0, s>>>(n, kk, vv, pw, f4, a4, wsum); break;
            case 4: k_fuse_runs4<4><<<grid, 256, 0, s>>>(n, kk, vv, pw, f4, a4, wsum); break;
            case 8: k_fuse_runs4<8><<<grid, 256, 0, s>>>(n, kk, vv, pw, f4, a4, wsum); break;
            case 16: k_fuse_runs4<16><<<grid, 256, 0, s>>>(n, kk, vv, pw, f4, a4, wsum); break;
            default: k_fuse_runs4<32><<<grid, 256, 0, s>>>(n, kk, vv, pw, f4, a4, wsum); break;
        }
    } else if (C <= 32) {
        k_fuse_runs<1><<<grid, 256, 0, s>>>(n, kk, vv, pw, f2d, C, acc, wsum);
    } else if (C <= 64) {
        k_fuse_runs<2><<<grid, 256, 0, s>>>(n, kk, vv, pw, f2d, C, acc, wsum);
    } else {
        k_fuse_runs<4><<<grid, 256, 0, s>>>(n, kk, vv, pw, f2d, C, acc, wsum);
    }
    count_launches(1);
    e = cudaGetLastError();
    // the sort's own wait flag: a run-out look-back left the slots unsorted and the sums wrong
    uint32_t flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, vmax + 1, sizeof(flag), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *sort_timeout = flag != 0;
    return e;
}

}  // namespace dv
