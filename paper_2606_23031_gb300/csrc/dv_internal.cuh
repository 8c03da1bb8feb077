// Internal types shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dv.h"

#define DV_TILE 16

// Per (view, octree) constants, computed on the host in double and rounded once.
struct OctParams {
    float A[9];          // unit camera-frame ray direction -> octree-local direction (R_i^T R_c)
    float Rw[9];         // octree-local -> world rotation (R_i), for voxel normals
    float M[9];          // octree-local point -> camera frame, rotation (R_c^T R_i)
    float m[3];          //   ... translation (R_c^T (t_i - t_c))
    float o_loc[3];      // camera centre in the octree's local frame (R_i^T (t_c - t_i))
    float clip_half[3];  // actor clip box half extents
    float root_min[3];   // center - root/2
    float root_size;
    int32_t role;
    int32_t sh_degree;
    int32_t max_level;
    int16_t rect[4];     // actor clip box tile rectangle [tx0, ty0, tx1, ty1] in the view (tx0 > tx1: off screen)
    int64_t O2[3];       // floor(2 * (o_loc - root_min) / root * 2^Lkey): BSP side tests in integers
    int64_t vox_offset;  // first voxel index of this octree within a view
    int64_t n_vox;
    const uint64_t* key;
    const float* dens;
    const float* sh;
};

// Per view (one camera of one render request).
struct ViewParams {
    int32_t W, H, tiles_x, tiles_y;
    float fx, fy, cx, cy;
    float near_, far_;
    float z_clip;        // camera-frame depth below which no ray sample can lie (near * min unit dz)
    int32_t tile_base;   // first global tile index of this view
    int64_t pix_base;    // first pixel of this view in the call's per-pixel arrays (upstream gradients, state)
    float* rgb;          // this view's outputs [H*W][3], [H*W], [H*W] (device)
    float* depth;
    float* alpha;
    float* normal;       // [H*W][3] normal state N (world frame), or null when normals are not rendered
};

// Shared by every kernel of a render call (passed by value).
struct BatchParams {
    int32_t n_view, n_oct;
    int32_t K;
    float inv_k;         // 1 / K
    float eps_stop;
    int32_t activation;
    int32_t Lkey;        // BSP key depth (max level over the octrees)
    int32_t oct_shift;   // 3 * Lkey
    int32_t view_shift;  // oct_shift + bits(n_oct)
    int32_t n_tiles;     // over all views
    int32_t n_tiles_large;  // tiles that 5 or more actor clip boxes cover (first in the tile order)
    int32_t n_tiles_small;  // tiles that 1 to 4 actor clip boxes cover (next in the tile order)
    int32_t normals;     // the call renders the normal state N (records carry voxel normals)
    int64_t n_vox;       // voxels of one view (all octrees)
    int64_t n_vis;       // visible (view, voxel)s = records of the call (set once the projection reports it)
    int64_t n_pairs;     // (tile, record) pairs of the call (likewise)
    int64_t vox_offset[DV_MAX_OCTREES + 1];
    int32_t tile_base[DV_MAX_VIEWS + 1];
    const ViewParams* views;  // device [n_view]
    const OctParams* octs;    // device [n_view][n_oct]
    const float4* nrm;        // device [n_vis]: voxel normal (world frame) of each record, when normals
    const uint32_t* sorted_g; // device [n_vis]: record -> view * n_vox + voxel
};

static_assert(sizeof(BatchParams) < 4096, "BatchParams is meant to stay small");

// 64-byte per-voxel render record, one per visible (view, voxel) in depth-key order.
//   v[0] = (min - o, size)   min corner relative to the camera centre o, both in the octree's frame
//   v[1] = (c0, c3, c1, c5)  the trilinear density as a polynomial in the voxel coordinates,
//   v[2] = (c2, c6, c4, c7)  rho = c0 + c1 x + c2 y + c3 z + c4 xy + c5 xz + c6 yz + c7 xyz, paired
//                            so that (c0, c3) + (c1, c5) x and (c2, c6) + (c4, c7) x are packed FMAs
//   v[3] = (r, g, b, 1/size)
struct __align__(16) VoxRec {
    float4 v[4];
};

// process-wide count of kernel launches issued by this library (all contexts)
namespace dv {

// Programmatic dependent launch.  The kernels of the rendering path are launched with
// programmatic stream serialisation: a kernel's blocks may be dispatched while the previous
// kernel of the stream drains.  Each of them starts with pdl_wait(), which returns once the
// previous kernel has completed and its memory is visible (a no-op for an ordinary launch), and
// then signals with pdl_launch_dependents() that the next kernel may be dispatched, which the
// hardware does only once every block of this grid has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
void count_launches(long long n);
}

// error flags written by kernels (bitmask in device memory)
#define DV_FLAG_BAD_LEVEL 1u
#define DV_FLAG_SPIN_TIMEOUT 2u  // a bounded wait of a sort ran out (folded in from the device's error word)

namespace dv {

struct Arena {
    cudaMemPool_t pool;
    cudaStream_t stream;
    void* ptrs[256];
    int n = 0;
    cudaError_t err = cudaSuccess;
    template <typename T>
    T* alloc(size_t count) {
        if (err != cudaSuccess) return nullptr;
        if (n >= 256) {
            err = cudaErrorMemoryAllocation;
            return nullptr;
        }
        void* p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        err = cudaMallocFromPoolAsync(&p, bytes, pool, stream);
        if (err != cudaSuccess) return nullptr;
        ptrs[n++] = p;
        return (T*)p;
    }
    void release() {
        for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], stream);
        n = 0;
    }
};

cudaError_t scan_u32_to_u64(const uint32_t* in, uint64_t* out, int64_t n, uint64_t* total_dev, Arena& ar,
                            cudaStream_t s);
cudaError_t scan_u32_to_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, Arena& ar,
                            cudaStream_t s);
// LSD radix sort of (key, value) pairs on bits [0, n_bits). Returns the buffers holding the result.
// call_err (device word, may be null): set to 1 if a bounded look-back wait of this sort ran out
// (the result is then not sorted); the device's wait-error word is set as well.
cudaError_t radix_sort_u64(uint64_t*& keys, uint32_t*& vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                           int n_bits, Arena& ar, cudaStream_t s, uint32_t* call_err = nullptr);
// streaming multiprocessors of the current device (cached per device)
int sm_count();
// test hook: one sort tile whose predecessor never publishes waits `spin_limit` reads and gives up;
// returns the tile's call flag and the device's wait-error word (which it then clears).  Synchronous.
cudaError_t debug_sort_timeout(int spin_limit, uint32_t* call_flag, uint32_t* device_flag, cudaStream_t s);

// Sort of n (key, value) pairs on bits [0, n_bits) whose digit counts the kernel that wrote the keys
// has already taken: hist[p][256] counts digit (key >> 8p) & 255 of every key, for every 8-bit pass p.
// `words` (sort_counted_words(n, n_bits) 32-bit words, zeroed by the caller) hold the passes' tile
// counters and look-back status.  keys/vals and keys_tmp/vals_tmp are the ping-pong buffers (the
// input is overwritten); the last pass writes vals_out and keys_out, or, with keys_out null, the
// ping-pong buffer it does not read, returned in keys_out.  call_err (device word, not null) is set
// to 1 if a bounded look-back wait runs out (the result is then not sorted).  Counts of 2^30 keys
// or more take reduce-then-scan passes (which count their own digits) and copy to the outputs.
int64_t sort_counted_words(int64_t n, int n_bits);
cudaError_t sort_counted_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_tmp, uint32_t* vals_tmp,
                             uint64_t*& keys_out, uint32_t* vals_out, int64_t n, int n_bits, const uint32_t* hist,
                             uint32_t* words, uint32_t* call_err, Arena& ar, cudaStream_t s);
cudaError_t sort_counted_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                             uint32_t*& keys_out, uint32_t* vals_out, int64_t n, int n_bits, const uint32_t* hist,
                             uint32_t* words, uint32_t* call_err, Arena& ar, cudaStream_t s);
// 8-bit passes of an n_bits key
int key_passes(int n_bits);

// kernel launchers (one thread per (view, voxel) unless stated)
// Projection: for each visible (view, voxel) g, cnt[g] (tiles) and rect[g] (pixel rectangle); the
// visible ones appended to (out_key, out_g) (depth key, g) in no particular order, the digits of
// their keys counted in key_hist [key_passes(key_bits)][256] (zeroed by the caller).  scal[4]
// (zeroed by the caller): visible count, pair count, flags (DV_FLAG_*), finished blocks; the last
// block copies the first three into host_out (mapped host memory), with the device's wait-error word
// (taken and cleared) folded into the flags, then writes `seq` into host_out[3] once the three are
// there.  It also clears work[5] (the call's work counters and sort flag).
cudaError_t launch_project(const BatchParams& bp, uint32_t* cnt, uint64_t* rect, uint64_t* out_key, uint32_t* out_g,
                           uint32_t* key_hist, int key_bits, unsigned long long* scal, uint64_t* host_out, uint64_t seq,
                           uint32_t* spin_err, unsigned long long* work, cudaStream_t s);
// copies n words into mapped host memory; with spin_err, takes (and clears) the device's wait-error
// word and sets DV_FLAG_SPIN_TIMEOUT in word flag_idx
cudaError_t launch_publish(const uint64_t* src, uint64_t* host_mapped_dst, int n, uint32_t* spin_err, int flag_idx,
                           cudaStream_t s);
// device address of this device's wait-error word (bounded waits that run out set it; shared by every
// context on the device); nullptr on failure
uint32_t* spin_error_word();
// One thread per visible voxel in depth order: records (and normals), rect_sorted, vis_start
// [n_view * n_oct + 1] (start of every (view, octree) group), and the (tile, record) pairs in
// depth order at offsets of a single-pass scan of the tile counts; counts the pairs of every tile in
// tile_cnt and the tile-sort digits in pair_hist [key_passes(tile_bits)][256].  tile_cnt, pair_hist,
// lb_status [records_emit_blocks(n_vis)] and ticket are zeroed by the caller.
cudaError_t launch_records_emit(const BatchParams& bp, const uint32_t* sorted_g, const uint64_t* sorted_key,
                                int64_t n_vis, int64_t n_pairs, const uint32_t* cnt, const uint64_t* rect,
                                VoxRec* rec, float4* nrm, uint64_t* rect_sorted, uint32_t* vis_start,
                                uint32_t* pair_key, uint32_t* pair_val, uint32_t* pair_hist, int tile_bits,
                                uint32_t* tile_cnt, unsigned long long* lb_status, uint32_t* ticket,
                                uint32_t* call_err, uint32_t* dev_err, cudaStream_t s);
int64_t records_emit_blocks(int64_t n_vis);
// per tile-sorted pair: its 8x4-block mask; per tile with pairs: its [first, end) range of the
// tile-sorted pair list; also copies *sort_err into the call's mapped status word
cudaError_t launch_pair_mask(const BatchParams& bp, const uint32_t* pair_key, const uint32_t* pair_val,
                             const uint64_t* rect_sorted, int64_t n_pairs, int64_t n_vis, uint8_t* mask,
                             uint2* tile_range, const uint64_t* sort_err, uint64_t* status_host, cudaStream_t s);
// the empty range for every tile without pairs, and the tiles ordered by decreasing list length (log2
// buckets of tile_cnt) within three groups, in this order: the tiles that 5 or more actor clip boxes
// cover (bp.n_tiles_large), those that 1 to 4 cover (bp.n_tiles_small), the others.  bucket: one byte
// of scratch per tile; scratch192: zeroed words.
cudaError_t launch_tile_order(const BatchParams& bp, const uint32_t* tile_cnt, int n_tiles, uint2* range,
                              uint8_t* bucket, uint32_t* scratch192, uint32_t* order, cudaStream_t s);
// Two more streams of the context with their events: a compositing pass runs its three launches (the
// tiles that many actor boxes cover, those that a few cover, the others) side by side on these and
// the call's stream.
struct Fork {
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
};

// outputs go to the views' buffers (ViewParams); n_seg and t_final per pixel are kept for the backward
cudaError_t launch_composite_fwd(const BatchParams& bp, const VoxRec* rec, const uint32_t* pair_val,
                                 const uint8_t* pair_mask, const uint2* tile_range, const uint32_t* vis_start,
                                 const uint32_t* tile_order, uint32_t* n_seg, float* t_final,
                                 unsigned long long* work, const Fork* fk, cudaStream_t s);
// with g_normal (the call rendered normals): gradient rows of 16 floats (8 densities, 3 colour, 3 normal, 2 pad),
// else of 12 (8 densities, 3 colour, 1 pad)
cudaError_t launch_composite_bwd(const BatchParams& bp, const VoxRec* rec, const uint32_t* pair_val,
                                 const uint8_t* pair_mask, const uint2* tile_range, const uint32_t* vis_start,
                                 const uint32_t* tile_order, const float* t_final, const float* g_rgb,
                                 const float* g_depth, const float* g_alpha, const float* g_normal, float* grad_rec,
                                 const Fork* fk, cudaStream_t s);
// replay of the forward that writes, for pixel p, the (voxel, weight T alpha) of each composited
// segment into slots [offsets[p], offsets[p+1]) (voxel index within the view's concatenated octrees)
cudaError_t launch_composite_export(const BatchParams& bp, const VoxRec* rec, const uint32_t* pair_val,
                                    const uint8_t* pair_mask, const uint2* tile_range, const uint32_t* vis_start,
                                    const uint32_t* tile_order, const int64_t* offsets, uint32_t* voxel, float* weight,
                                    const Fork* fk, cudaStream_t s);
cudaError_t launch_sh_bwd(const BatchParams& bp, const uint32_t* sorted_g, int64_t n_vis, const VoxRec* rec,
                          const float* grad_rec, bool with_normals, float* const* d_dens, float* const* d_sh,
                          cudaStream_t s);

// feature fields over a weights export (see dv_features.cu)
cudaError_t launch_feat_render(int64_t n_pix, const int64_t* off, const uint32_t* vox, const float* wgt,
                               const float* feat, int C, float* out, cudaStream_t s);
// one launch, no scratch and no synchronisation (chunks of consecutive pixels grouped in shared memory)
cudaError_t feat_fuse(int64_t n_pix, const int64_t* off, const uint32_t* vox, const float* wgt, const float* f2d,
                      int C, float* acc, float* wsum, cudaStream_t s);

// LiDAR-guided initialisation (see dv_init.cu); the calls that return a size synchronise the stream.
// The calls that sort set *sort_timeout (host) when the sort's bounded wait ran out; they synchronise
// the stream before they return.
cudaError_t key_levels(const uint64_t* keys, int64_t n, uint32_t* levels_host, Arena& ar, cudaStream_t s);
cudaError_t shared_corners(const uint64_t* keys, int64_t n, int max_level, uint64_t* grid_out, uint32_t* index_out,
                           int64_t* n_corners, Arena& ar, cudaStream_t s, bool* sort_timeout);
cudaError_t soft_prior(const uint64_t* grid, int64_t n_corners, const double* center, double root_size, int max_level,
                       const float* cloud, int64_t m, float s_min, float v_close, float v_far, float* dens, Arena& ar,
                       cudaStream_t s, bool* sort_timeout);
cudaError_t subdivide_round(const uint64_t* keys, int64_t n, const double* center, double root_size, int max_level,
                            const float* cloud, int64_t m, float thr, uint64_t* out, int64_t* n_out, Arena& ar,
                            cudaStream_t s, bool* sort_timeout);
// uniform leaf grid of an actor (Sec. 3.3, assets): keys of the 8^level leaves (i fastest) and every
// corner density set to v_init
cudaError_t asset_grid(int level, float v_init, uint64_t* keys, float* dens, cudaStream_t s);
// a camera of the visibility pruning (double precision, camera -> world rotation row-major)
struct InitCam {
    double R[9], t[3];
    double fx, fy, cx, cy, near_, far_;
    int32_t W, H;
};
cudaError_t visibility_prune(const uint64_t* keys, int64_t n, const double* center, double root_size,
                             const InitCam* cams_host, int n_cam, double z_min, uint64_t* out, int64_t* n_out,
                             Arena& ar, cudaStream_t s);
cudaError_t corner_gather(const uint32_t* index, int64_t n, const float* corner, float* dens, cudaStream_t s);
cudaError_t corner_scatter(const uint32_t* index, int64_t n, const float* d_dens, float* d_corner, cudaStream_t s);

// one camera of a sky composite: camera -> world rotation (row-major) and intrinsics
struct SkyView {
    float R[9];
    float fx, fy, cx, cy;
    int32_t W, H;
};
cudaError_t launch_sky_fwd(const SkyView& v, const float* env, int He, int We, const float* rgb, const float* alpha,
                           float* out, cudaStream_t s);
cudaError_t launch_sky_bwd(const SkyView& v, const float* env, int He, int We, const float* alpha, const float* d_out,
                           float* d_env, float* d_alpha, cudaStream_t s);

// camera and pose checks of one render request (the same as dv_render's); no context needed
dv_status validate_request(const dv_camera& cam, const dv_pose* poses, int n_oct);

// device memory a render call takes from its context's pool: the part known before any work is
// enqueued (n_view views of n_oct octrees, NT = views x voxels, tiles and pixels over the views) and
// the part that follows from the projection's sizes (visible voxels, pairs)
int64_t render_need_before(int64_t n_view, int64_t n_oct, int64_t NT, int64_t tiles, int64_t pix);
int64_t render_need_after(int64_t n_vis, int64_t P, int64_t tiles, int key_bits, int tile_bits, bool normals);

// render of views whose outputs live in separate device buffers (serving loop); the saved state
// (non-null) lets the caller check the call's sorts once its stream has finished
dv_status render_views_into(dv_ctx* ctx, const dv_octree* oct, int n_oct, const dv_view* views, int n_view,
                            const dv_opts* opts, float* const* rgbs, float* const* depths, float* const* alphas,
                            dv_state** saved, void* stream);

}  // namespace dv
