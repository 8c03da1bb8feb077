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
// atomic rate (one add per slot and channel), so the slots of a chunk of consecutive pixels are
// grouped by voxel in shared memory and each voxel's sum over the chunk is added once.
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

// ---- fusion by pixel chunks ----
// A block takes FL_PIX consecutive pixels (their slots are one contiguous range) and a slice of up
// to FL_SW channels.  Neighbouring pixels see mostly the same voxels (a 128-pixel run of an image
// row: a few thousand slots over about a hundred distinct voxels), so the block sums the chunk's
// slots per voxel and adds each voxel's sums to the global rows once per chunk.  The 2-D features
// are read once, in order, and the slots need no global sort.
//  * The chunk's 2-D feature slice is staged in shared memory.
//  * The slots, FL_PIECE at a time, get a row from an open-addressing table keyed by the voxel
//    index (compare-and-swap inserts, FL_ROWS rows); a voxel that finds no row within FL_PROBES
//    probes goes to the overflow row, whose slots are added to the global sums one by one.
//  * A counting sort by row groups the piece's slots and lists the rows that hold any; warp w takes
//    listed rows w, w + 8, ...: its four 8-lane groups walk every fourth slot of the row, a lane
//    holding two 4-channel quads of the sums in registers, and the groups' sums are added by
//    shuffles before one atomic add per quad.
constexpr int FL_PIX = 128;     // pixels per chunk
constexpr int FL_SW = 64;       // channels per slice (16 quads)
constexpr int FL_ROWS = 1023;   // voxel rows; row FL_ROWS holds the overflow slots
constexpr int FL_TE = FL_ROWS + 1;  // table entries, FL_TE / FL_THREADS per thread in the scan
constexpr int FL_PIECE = 3072;  // slots grouped at once (three 70 KB blocks fit an SM)
constexpr int FL_PROBES = 32;
constexpr int FL_THREADS = 256;
constexpr int FL_SPT = FL_PIECE / FL_THREADS;  // slots per thread and piece
constexpr uint32_t FL_EMPTY = 0xffffffffu;

struct FuseSmem {
    float4 f[FL_PIX][FL_SW / 4];      // 2-D features of the chunk's pixels, this slice
    int64_t off[FL_PIX + 1];          // slot offsets of the chunk's pixels
    uint32_t key[FL_ROWS];            // voxel of each row (FL_EMPTY: free)
    uint32_t cnt[FL_TE];              // slots per row, then the fill cursors
    uint32_t start[FL_TE + 1];        // first grouped slot of each row
    uint16_t occ[FL_TE];              // the rows that hold slots, in row order
    uint32_t n_occ;
    uint32_t wtot[FL_THREADS / 32];   // scan: warp totals (slots, then rows)
    uint32_t wocc[FL_THREADS / 32];
    float sw[FL_PIECE];               // grouped by row: the slot's weight,
    uint16_t order[FL_PIECE];         //   its index in the piece,
    uint8_t spl[FL_PIECE];            //   and its pixel within the chunk
};

__device__ __forceinline__ uint32_t fl_hash(uint32_t v) { return ((v * 2654435761u) >> 16) % FL_ROWS; }

// 16-byte asynchronous global -> shared copy (L2 only) and its fences
__device__ __forceinline__ void fl_cp_async16(void* smem, const void* gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void fl_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void fl_cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void fl_add4(float4& a, float w, float4 f) {
    a.x = fmaf(w, f.x, a.x);
    a.y = fmaf(w, f.y, a.y);
    a.z = fmaf(w, f.z, a.z);
    a.w = fmaf(w, f.w, a.w);
}

// adds quad a (channels c .. c + 3, those below C) into row v of the global sums
template <bool VEC>
__device__ __forceinline__ void fl_flush4(float* __restrict__ acc, uint32_t v, int C, int c, float4 a) {
    if (c >= C || (a.x == 0.0f && a.y == 0.0f && a.z == 0.0f && a.w == 0.0f)) return;
    float* row = acc + (size_t)v * C + c;
    if (VEC) {
        atomicAdd(reinterpret_cast<float4*>(row), a);
    } else {
        atomicAdd(row, a.x);
        if (c + 1 < C) atomicAdd(row + 1, a.y);
        if (c + 2 < C) atomicAdd(row + 2, a.z);
        if (c + 3 < C) atomicAdd(row + 3, a.w);
    }
}

template <bool VEC>
__global__ void __launch_bounds__(FL_THREADS, 3) k_fuse_local(int64_t n_pix, const int64_t* __restrict__ off,
                                                             const uint32_t* __restrict__ vox,
                                                             const float* __restrict__ wgt,
                                                             const float* __restrict__ f2d, int C,
                                                             float* __restrict__ acc, float* __restrict__ wsum) {
    extern __shared__ __align__(16) unsigned char fl_raw[];
    FuseSmem& S = *reinterpret_cast<FuseSmem*>(fl_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q0 = 2 * (lane & 7), g = lane >> 3;  // first of the lane's two channel quads, 8-lane group
    for (int i = tid; i < FL_ROWS; i += FL_THREADS) S.key[i] = FL_EMPTY;
    const int64_t n_chunks = (n_pix + FL_PIX - 1) / FL_PIX;
    const int n_slices = (C + FL_SW - 1) / FL_SW;
    for (int64_t task = blockIdx.x; task < n_chunks * n_slices; task += gridDim.x) {
        const int64_t p0 = (task / n_slices) * FL_PIX;
        const int c0 = (int)(task % n_slices) * FL_SW;
        const int np = (int)min((int64_t)FL_PIX, n_pix - p0);
        __syncthreads();  // the previous task is done with the shared arrays
        // the chunk's 2-D feature slice: 16-byte asynchronous copies (rows 16-byte aligned), which
        // land while the slots are grouped; otherwise plain loads
        if (VEC) {
            for (int i = tid; i < FL_PIX * (FL_SW / 4); i += FL_THREADS) {
                const int pl = i / (FL_SW / 4), qd = i % (FL_SW / 4), c = c0 + 4 * qd;
                if (pl < np && c < C)
                    fl_cp_async16(&S.f[pl][qd], f2d + (size_t)(p0 + pl) * C + c);
                else
                    S.f[pl][qd] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            fl_cp_async_commit();
        } else {
            for (int i = tid; i < FL_PIX * FL_SW; i += FL_THREADS) {
                const int pl = i / FL_SW, j = i % FL_SW, c = c0 + j;
                (&S.f[0][0].x)[i] = pl < np && c < C ? __ldg(f2d + (size_t)(p0 + pl) * C + c) : 0.0f;
            }
        }
        for (int i = tid; i <= np; i += FL_THREADS) S.off[i] = off[p0 + i];
        __syncthreads();
        const int64_t e_end = S.off[np];
        for (int64_t e0 = S.off[0]; e0 < e_end; e0 += FL_PIECE) {
            const int ns = (int)min((int64_t)FL_PIECE, e_end - e0);
            for (int i = tid; i < FL_TE; i += FL_THREADS) S.cnt[i] = 0;
            // this thread's slots tid + j * FL_THREADS: loads first (all in flight together)
            uint32_t v_[FL_SPT], r_[FL_SPT];
            float w_[FL_SPT];
#pragma unroll
            for (int j = 0; j < FL_SPT; ++j) {
                const int k = tid + j * FL_THREADS;
                v_[j] = k < ns ? __ldg(vox + e0 + k) : 0u;
                w_[j] = k < ns ? __ldg(wgt + e0 + k) : 0.0f;
            }
            __syncthreads();
            // each slot's pixel (binary search of the chunk's offsets) and its voxel's row
#pragma unroll
            for (int j = 0; j < FL_SPT; ++j) {
                const int k = tid + j * FL_THREADS;
                r_[j] = 0u;
                if (k < ns) {
                    const int64_t e = e0 + k;
                    int lo = 0, hi = np - 1;  // the owner i has off[i] <= e < off[i + 1]
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (S.off[mid] <= e)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    uint32_t h = fl_hash(v_[j]), row = FL_ROWS;
                    for (int probe = 0; probe < FL_PROBES; ++probe) {
                        const uint32_t old = atomicCAS(&S.key[h], FL_EMPTY, v_[j]);
                        if (old == FL_EMPTY || old == v_[j]) {
                            row = h;
                            break;
                        }
                        h = h + 1 == FL_ROWS ? 0u : h + 1;
                    }
                    r_[j] = ((uint32_t)lo << 16) | row;
                    atomicAdd(&S.cnt[row], 1u);
                }
            }
            __syncthreads();
            // exclusive scan of the FL_TE row counts (FL_TE / FL_THREADS consecutive entries per thread),
            // and the list of the rows that hold slots
            {
                constexpr int EPT = FL_TE / FL_THREADS;
                uint32_t c[EPT], sum = 0, nocc = 0;
#pragma unroll
                for (int t = 0; t < EPT; ++t) {
                    c[t] = S.cnt[tid * EPT + t];
                    sum += c[t];
                    nocc += c[t] ? 1u : 0u;
                }
                uint32_t inc = sum, ino = nocc;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
                    const uint32_t z = __shfl_up_sync(0xffffffffu, ino, d);
                    if (lane >= d) {
                        inc += y;
                        ino += z;
                    }
                }
                if (lane == 31) {
                    S.wtot[warp] = inc;
                    S.wocc[warp] = ino;
                }
                __syncthreads();
                uint32_t base = inc - sum, bo = ino - nocc;
                for (int w = 0; w < warp; ++w) {
                    base += S.wtot[w];
                    bo += S.wocc[w];
                }
#pragma unroll
                for (int t = 0; t < EPT; ++t) {
                    const int r = tid * EPT + t;
                    S.start[r] = base;
                    S.cnt[r] = 0;
                    if (c[t]) S.occ[bo++] = (uint16_t)r;
                    base += c[t];
                }
                if (tid == FL_THREADS - 1) {
                    S.start[FL_TE] = base;
                    S.n_occ = bo;
                }
            }
            __syncthreads();
            // group the slots by row
#pragma unroll
            for (int j = 0; j < FL_SPT; ++j) {
                const int k = tid + j * FL_THREADS;
                if (k < ns) {
                    const uint32_t row = r_[j] & 0xffffu;
                    const uint32_t pos = S.start[row] + atomicAdd(&S.cnt[row], 1u);
                    S.sw[pos] = w_[j];
                    S.order[pos] = (uint16_t)k;
                    S.spl[pos] = (uint8_t)(r_[j] >> 16);
                }
            }
            if (VEC && e0 == S.off[0]) fl_cp_async_wait_all();  // the feature slice has landed
            __syncthreads();
            // per row with slots: the warp's four 8-lane groups take every fourth slot, a lane holding
            // two 4-channel quads (q0, q0 + 1) of the sums in registers
            const uint32_t n_occ = S.n_occ;
            for (uint32_t oi = warp; oi < n_occ; oi += FL_THREADS / 32) {
                const uint32_t r = S.occ[oi];
                const uint32_t s0 = S.start[r], s1 = S.start[r + 1];
                if (r < FL_ROWS) {
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                    float ws = 0.0f;
#pragma unroll 2
                    for (uint32_t i = s0 + g; i < s1; i += 4) {
                        const float wv = S.sw[i];
                        const float4* fr = S.f[S.spl[i]];
                        fl_add4(a, wv, fr[q0]);
                        fl_add4(b, wv, fr[q0 + 1]);
                        ws += wv;
                    }
#pragma unroll
                    for (int d = 8; d < 32; d <<= 1) {
                        a.x += __shfl_xor_sync(0xffffffffu, a.x, d);
                        a.y += __shfl_xor_sync(0xffffffffu, a.y, d);
                        a.z += __shfl_xor_sync(0xffffffffu, a.z, d);
                        a.w += __shfl_xor_sync(0xffffffffu, a.w, d);
                        b.x += __shfl_xor_sync(0xffffffffu, b.x, d);
                        b.y += __shfl_xor_sync(0xffffffffu, b.y, d);
                        b.z += __shfl_xor_sync(0xffffffffu, b.z, d);
                        b.w += __shfl_xor_sync(0xffffffffu, b.w, d);
                        ws += __shfl_xor_sync(0xffffffffu, ws, d);
                    }
                    const uint32_t v = S.key[r];
                    if (g == 0) {
                        fl_flush4<VEC>(acc, v, C, c0 + 4 * q0, a);
                        fl_flush4<VEC>(acc, v, C, c0 + 4 * q0 + 4, b);
                    }
                    if (lane == 0 && wsum && c0 == 0 && ws != 0.0f) atomicAdd(wsum + v, ws);
                } else {
                    // overflow row: every slot added on its own
                    for (uint32_t i = s0 + g; i < s1; i += 4) {
                        const float wv = S.sw[i];
                        const uint32_t v = __ldg(vox + e0 + S.order[i]);
                        const float4* fr = S.f[S.spl[i]];
                        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                        fl_add4(a, wv, fr[q0]);
                        fl_add4(b, wv, fr[q0 + 1]);
                        fl_flush4<VEC>(acc, v, C, c0 + 4 * q0, a);
                        fl_flush4<VEC>(acc, v, C, c0 + 4 * q0 + 4, b);
                        if (q0 == 0 && wsum && c0 == 0 && wv != 0.0f) atomicAdd(wsum + v, wv);
                    }
                }
            }
            __syncthreads();
            for (int i = tid; i < FL_ROWS; i += FL_THREADS) S.key[i] = FL_EMPTY;
        }
        if (VEC) fl_cp_async_wait_all();  // a chunk without slots: no copy outlives the task
    }
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
                      int C, float* acc, float* wsum, cudaStream_t s) {
    if (n_pix <= 0 || C <= 0) return cudaSuccess;
    const int64_t n_chunks = (n_pix + FL_PIX - 1) / FL_PIX;
    const int64_t tasks = n_chunks * ((C + FL_SW - 1) / FL_SW);
    const int64_t cap = (int64_t)sm_count() * 3;  // three 66 KB blocks per SM
    const unsigned grid = (unsigned)(tasks < cap ? tasks : cap);
    const size_t smem = sizeof(FuseSmem);
    // 16-byte copies of the 2-D features and vector atomics need 16-byte aligned rows of both arrays
    const bool vec = C % 4 == 0 && ((reinterpret_cast<uintptr_t>(acc) | reinterpret_cast<uintptr_t>(f2d)) & 15) == 0;
    cudaError_t e;
    if (vec) {
        e = cudaFuncSetAttribute(k_fuse_local<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) k_fuse_local<true><<<grid, FL_THREADS, smem, s>>>(n_pix, off, vox, wgt, f2d, C, acc, wsum);
    } else {
        e = cudaFuncSetAttribute(k_fuse_local<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) k_fuse_local<false><<<grid, FL_THREADS, smem, s>>>(n_pix, off, vox, wgt, f2d, C, acc, wsum);
    }
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dv
