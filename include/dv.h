/*
 * dv.h -- C ABI of the GB300 compositional sparse-voxel rasterizer.
 *
 * The library renders one static background octree plus any number of rigid
 * actor octrees in a single pass and back-propagates through that pass
 * (DrivingVoxels, Sec. 3.4 and Algorithm 1 of the supplement):
 *
 *   dv_render           octrees[], poses[], cameras[] -> RGB, depth, alpha
 *   dv_render_backward  dL/dRGB, dL/ddepth, dL/dalpha -> dL/d corner densities,
 *                       dL/d SH coefficients
 *
 * Everything on the compute path runs in this library's sm_103a kernels; the
 * caller only supplies device buffers and a CUDA stream.  No function throws;
 * every fallible call returns a dv_status and, on failure, leaves a message
 * retrievable with dv_last_error().
 *
 * Conventions shared by every call
 *  - Pointers named "device" are CUDA device pointers on the context's device;
 *    the caller owns them and keeps them alive until the work enqueued on the
 *    given stream has finished.  Structs passed by host pointer are read
 *    during the call only.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All work is enqueued on it.  A render call waits once on the host for the
 *    sizes its projection kernel reports (an event, not a stream
 *    synchronisation) to size its buffers: the only host wait on the path.
 *  - Leaf keys: bits [0,19) = i, [19,38) = j, [38,57) = k, [57,62) = level.
 *    A leaf spans min = center - root_size/2 + (i,j,k) * s to min + s with
 *    s = root_size / 2^level, in its octree's local frame (Sec. 3.1, where each
 *    leaf is stored as a level and an integer grid index).
 *  - Corner c of the 8 densities sits at offset (c&1, (c>>1)&1, (c>>2)&1).
 *  - Cameras use OpenCV axes (x right, y down, z forward); pixel (u,v) casts
 *    the ray through (u+0.5, v+0.5); depth is distance along the unit ray.
 *  - Output images are row-major [H][W] (RGB: [H][W][3]); for several
 *    cameras the images are concatenated in camera order.
 *
 * Thread safety: a context may be used by one host thread at a time.  Distinct
 * contexts are independent.
 */
#ifndef DV_H
#define DV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DV_OK = 0,
    DV_ERR_INVALID_ARG = 1,  /* a size, pointer, level or option is out of range */
    DV_ERR_INVALID_POSE = 2, /* a rotation is not orthonormal with det +1 (tol 1e-5) */
    DV_ERR_CAPACITY = 3,     /* a size exceeds the library's fixed limits */
    DV_ERR_CUDA = 4,         /* a CUDA runtime call failed (message has the CUDA error) */
    DV_ERR_TIMEOUT = 5,      /* a bounded wait ran out (a sort's look-back, or a serving wait) */
    DV_ERR_NOMEM = 6         /* device or host allocation failed */
} dv_status;

enum { DV_ROLE_BG = 0, DV_ROLE_ACTOR = 1 };
enum { DV_ACT_EXPLIN = 0, DV_ACT_IDENTITY = 1 };

#define DV_MAX_OCTREES 128   /* background + up to 127 actors per call */
#define DV_MAX_VIEWS 64      /* views (cameras / requests) per render call */
#define DV_MAX_LEVEL 16      /* deepest leaf level accepted */
#define DV_MAX_IMAGE 16384   /* maximum W and H */
#define DV_MAX_SH_DEGREE 3

typedef struct dv_ctx dv_ctx;
typedef struct dv_state dv_state;

/* One octree (Sec. 3.1 background, Sec. 3.2 actor in its canonical frame). */
typedef struct {
    int64_t n_vox;          /* number of leaves (>= 0, < 2^31 summed over a call) */
    int32_t sh_degree;      /* 0..3 */
    int32_t role;           /* DV_ROLE_BG for octree 0, DV_ROLE_ACTOR for the others */
    int32_t max_level;      /* upper bound on the leaf levels present (0..16); a larger
                               level found on the device fails the call */
    int32_t reserved;
    double center[3];       /* AABB centre (local frame) */
    double root_size;       /* AABB edge length (local frame) */
    float clip_half[3];     /* actor: clip box half extents around the local origin;
                               the actor owns the ray interval inside this box
                               (Sec. 3.4); ignored for the background */
    const uint64_t* key;    /* device [n_vox] leaf keys (borrowed) */
    const float* dens;      /* device [n_vox][8] raw corner densities (borrowed) */
    const float* sh;        /* device [n_vox][(deg+1)^2][3] SH coefficients (borrowed) */
} dv_octree;

/* Rigid transform local -> world, p_w = R p_l + t, R row-major (Sec. 3.2 T_t^i). */
typedef struct {
    float R[9];
    float t[3];
} dv_pose;

typedef struct {
    int32_t W, H;           /* image size in pixels (0 allowed: nothing rendered) */
    float fx, fy, cx, cy;   /* pinhole intrinsics (fx, fy > 0) */
    dv_pose cam_to_world;   /* camera pose */
    float near_, far_;      /* ray distance range, 0 < near < far */
} dv_camera;

/* One view of a batched render: a camera and the poses of every octree for it
 * (its own timestamp).  `poses` is a host array [n_oct] read during the call. */
typedef struct {
    dv_camera camera;
    const dv_pose* poses;
} dv_view;

typedef struct {
    int32_t K;              /* midpoint samples per voxel segment, 1..16 */
    float eps_stop;         /* stop a ray once its transmittance drops below this (Alg. 1) */
    int32_t activation;     /* DV_ACT_EXPLIN (default) or DV_ACT_IDENTITY */
    int32_t reserved;
} dv_opts;

/* Creates a context on CUDA device `device`.  The context owns a stream-ordered
 * memory pool for the library's scratch; *ctx is NULL on failure. */
dv_status dv_create(dv_ctx** ctx, int32_t device);
void dv_destroy(dv_ctx* ctx);
/* Message of the last failing call on this context ("" if none). */
const char* dv_last_error(const dv_ctx* ctx);
/* Library version string. */
const char* dv_version(void);
/*
 * Bounded waits.  The one-sweep radix sort's look-back is the library's only
 * wait on other thread blocks (it waits only on tiles that started earlier, so
 * it ends); each spin is bounded, and a bound that runs out marks two words:
 *  - the call's own flag.  Calls that sort and synchronise anyway (feature
 *    fusion, the initialisation calls) read it before they return and fail
 *    with DV_ERR_TIMEOUT.  A render publishes it, after its last sort, into a
 *    host word of its saved state: dv_state_check reports it, the backward of
 *    that state refuses to run once it is known, and the serving loop fails
 *    the batch's requests.
 *  - a device-wide word shared by every context on the device (a sticky
 *    fallback for a timeout nobody checked): the next dv_render on the device
 *    takes and clears it in its size read-back and fails with DV_ERR_TIMEOUT.
 * dv_debug_flag_spin_timeout sets the device word from the host, so the
 * fallback path can be checked.  Synchronous.
 */
dv_status dv_debug_flag_spin_timeout(dv_ctx* ctx);

/*
 * Test hook of the bounded wait itself: launches one tile of a sort pass
 * whose predecessor tile never publishes, with at most `spin_limit` reads
 * (1 .. 2^20) per wait, and returns the tile's call flag and the device-wide
 * word as the kernel left them (both 1 when the wait ran out), then clears the
 * device-wide word.  Synchronous; the kernel ends after its bounded waits.
 */
dv_status dv_debug_sort_timeout(dv_ctx* ctx, int32_t spin_limit, uint32_t* call_flag, uint32_t* device_flag);

/*
 * Workspace reservation (the CAPACITY contract).  By default a context takes
 * whatever scratch a call needs from its pool.  dv_reserve(ctx, bytes) limits
 * each render call to `bytes` of workspace (its saved state plus its scratch)
 * and grows the pool to that size now, so calls within the reservation do not
 * allocate new device memory; bytes = 0 removes the limit.  A render that needs
 * more fails with DV_ERR_CAPACITY, either before any work is enqueued (the part
 * that follows from the octree, camera and tile counts) or after the
 * projection reported its sizes (visible voxels and pairs; the outputs are then
 * untouched).  dv_workspace_need returns the bytes the last render needed, or
 * the part known when it failed: reserve that and retry (a second failure, if
 * any, then reports the whole need).  DV_ERR_NOMEM if the device cannot hold
 * the reservation.
 */
dv_status dv_reserve(dv_ctx* ctx, int64_t bytes);
dv_status dv_workspace_need(const dv_ctx* ctx, int64_t* bytes);

/*
 * Asset initialisation (Sec. 3.3, "Assets"): the octree of a new actor is a
 * uniform leaf grid in its canonical frame (origin at the centre of its 3-D
 * box, axes along the box's), whose cubic bound is the largest box dimension
 * scaled by 1.2, with every corner density at one value (the paper's -10,
 * empty space, for every size and category).
 *   box_dims[3]   host, the box's dimensions (> 0, any order of axes)
 *   level         leaf level of the grid, 0..10 (8^level leaves)
 *   capacity      leaves keys/dens can hold; DV_ERR_CAPACITY below 8^level,
 *                 before any work is enqueued
 *   keys, dens    device outputs [8^level] (layout of dv_octree: leaf (i, j, k)
 *                 at index (k 2^level + j) 2^level + i) and [8^level][8]
 *                 (16-byte aligned), every entry v_init
 *   root_size     host output: 1.2 * max(box_dims); the grid's centre is the
 *                 local origin (0, 0, 0)
 *   n_leaves      host output: 8^level
 * The SH coefficients are the caller's (zero gives a colour of 0.5 grey).
 */
dv_status dv_asset_init(dv_ctx* ctx, const float* box_dims, int32_t level, float v_init, int64_t capacity,
                        uint64_t* keys, float* dens, double* root_size, int64_t* n_leaves, void* stream);

/*
 * Forward render (Sec. 3.4, Algorithm 1).  For each pixel of each camera the
 * ray is split into background and actor intervals by the actor clip boxes
 * (the box entered first owns any overlap), and every interval is composited
 * front to back from its octree's voxels with transmittance carried across
 * the borders; a ray stops once T < opts->eps_stop.
 *
 *   oct[n_oct], poses[n_oct]  host arrays; oct[0] is the background (its pose
 *                             places it in the world, normally identity)
 *   cams[n_cam]               host array
 *   rgb, depth, alpha         device outputs, concatenated per camera:
 *                             rgb [sum H*W][3], depth/alpha [sum H*W]; alpha = 1 - T
 *   saved                     if non-NULL, receives a state for
 *                             dv_render_backward (free it with dv_state_free);
 *                             the state borrows rgb/depth/alpha and the octree
 *                             buffers: they must stay unchanged until it is freed
 * Errors: DV_ERR_INVALID_ARG / DV_ERR_INVALID_POSE / DV_ERR_CAPACITY before any
 * work is enqueued; DV_ERR_CUDA or DV_ERR_INVALID_ARG (a leaf level above its
 * octree's max_level) after; the outputs are then undefined.
 */
dv_status dv_render(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_pose* poses, const dv_camera* cams,
                    int32_t n_cam, const dv_opts* opts, float* rgb, float* depth, float* alpha, dv_state** saved,
                    void* stream);

/*
 * Batched render of independent views (same method as dv_render): every view
 * has its own camera and its own octree poses (e.g. requests at different
 * timestamps), and all views go through one launch per stage, with the tiles of
 * every view scheduled together.  Up to DV_MAX_VIEWS views; outputs are
 * concatenated in view order as for dv_render; `saved` covers all views.
 */
dv_status dv_render_views(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_view* views, int32_t n_view,
                          const dv_opts* opts, float* rgb, float* depth, float* alpha, dv_state** saved,
                          void* stream);

/*
 * Backward of dv_render (the gradient passes through every voxel segment, Sec. 3.4).
 * Given dL/dRGB [sum H*W][3], dL/ddepth and dL/dalpha [sum H*W] (device; any of
 * the three may be NULL = zero), ADDS dL/d dens into d_dens[i] ([n_vox][8]) and
 * dL/d SH into d_sh[i] ([n_vox][nsh][3]) for every octree i (host arrays of
 * device pointers; an entry may be NULL to skip that octree).  The replay
 * follows the forward's segments exactly, including its early stop.
 * Summation order of the per-voxel gradient sums is not fixed (atomics).
 */
dv_status dv_render_backward(dv_ctx* ctx, dv_state* state, const float* d_rgb, const float* d_depth,
                             const float* d_alpha, float* const* d_dens, float* const* d_sh, void* stream);

/*
 * dv_render plus the normal state N of Algorithm 1 (Sec. 3.4: the pixel state
 * also sums voxel normals): N = sum over the composited segments of
 * T_k alpha_k n_k, with n the voxel's normal in world coordinates -- minus the
 * normalised gradient of the voxel's trilinear raw density at its centre
 * (per axis: the four corners on the high side minus the four on the low
 * side), rotated by its octree's pose; zero where that gradient vanishes.  N is
 * not normalised (compare with N / |N|, as the normal loss of the paper does).
 *   normal   device output [sum H*W][3], concatenated per camera like rgb
 * Other arguments, errors and the saved state as for dv_render; the state also
 * borrows `normal`.
 */
dv_status dv_render_normals(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_pose* poses,
                            const dv_camera* cams, int32_t n_cam, const dv_opts* opts, float* rgb, float* depth,
                            float* alpha, float* normal, dv_state** saved, void* stream);

/*
 * Backward of dv_render_normals: as dv_render_backward, plus dL/dN
 * (d_normal, device [sum H*W][3], world frame; NULL = zero), which reaches the
 * corner densities both through the compositing weights and through each
 * voxel's normal.  DV_ERR_INVALID_ARG if `state` comes from a call without
 * normals and d_normal is non-NULL.
 */
dv_status dv_render_backward_normals(dv_ctx* ctx, dv_state* state, const float* d_rgb, const float* d_depth,
                                     const float* d_alpha, const float* d_normal, float* const* d_dens,
                                     float* const* d_sh, void* stream);

/* Releases a saved state (stream-ordered on the stream of its render call). */
void dv_state_free(dv_state* state);

/* DV_ERR_TIMEOUT if a sort of the state's render ran out of its bounded wait
 * (the state's results are then invalid), else DV_OK.  With wait = 0 it only
 * reads what the render has published so far (DV_OK while unknown); with
 * wait != 0 it first synchronises the state's stream. */
dv_status dv_state_check(const dv_state* state, int32_t wait);

/*
 * Compositing weights of a saved render, for feature fields (Sec. 4, "3D
 * Semantic Segmentation": RGB accumulation with the colour replaced by a
 * per-voxel feature, and 2-D features fused into the voxels).  For pixel p
 * (concatenated over the call's views like rgb), the segments the forward
 * composited, with voxel index v (within the concatenation of the octrees in
 * call order: octree o's voxel j is sum_{i<o} n_vox_i + j) and weight
 * w = T alpha, so that RGB = sum w c(v) and alpha = sum w.  A voxel cut by an
 * actor box can appear twice in one pixel's list.
 *
 * dv_state_weight_offsets: writes the exclusive prefix of the per-pixel segment
 * counts to offsets ([sum H*W + 1], device; pixel p owns slots
 * [offsets[p], offsets[p+1])) and the total to *total (host).  Synchronises the
 * stream.
 * dv_state_weights: fills voxel[total] and weight[total] (device).  The replay
 * uses the forward's arithmetic and stop rule, so it fills exactly the counted
 * slots.
 */
dv_status dv_state_weight_offsets(dv_ctx* ctx, dv_state* state, int64_t* offsets, int64_t* total, void* stream);
dv_status dv_state_weights(dv_ctx* ctx, dv_state* state, const int64_t* offsets, uint32_t* voxel, float* weight,
                           void* stream);

/*
 * Feature render over a weights export: out[p][c] = sum over p's slots of
 * weight * feat[voxel][c], for C channels (feat device [n_voxels][C], out
 * device [n_pix][C]; voxel indices must be < the rows of feat).
 */
dv_status dv_features_render(dv_ctx* ctx, int64_t n_pix, const int64_t* offsets, const uint32_t* voxel,
                             const float* weight, const float* feat, int32_t C, float* out, void* stream);

/*
 * Feature fusion over a weights export (the transpose of dv_features_render):
 * ADDS weight * feat2d[p][c] into accum[voxel][c] and weight into wsum[voxel]
 * (NULL = skip) for every slot of every pixel; accum / wsum is then the
 * weighted mean of the 2-D features seen by each voxel.  One kernel: the
 * slots of every 128 consecutive pixels are grouped by voxel in shared memory
 * and each voxel's sum over them is added once per channel (atomics, so the
 * order of the additions varies from run to run).  Allocates nothing and does
 * not synchronise the stream.
 */
dv_status dv_features_fuse(dv_ctx* ctx, int64_t n_pix, const int64_t* offsets, const uint32_t* voxel,
                           const float* weight, const float* feat2d, int32_t C, float* accum, float* wsum,
                           void* stream);

/*
 * LiDAR-guided initialisation of the background octree (Sec. 3.3).  Keys use
 * the leaf layout of dv_octree (level << 57 | k << 38 | j << 19 | i); every
 * call that returns a size synchronises the stream.
 *
 * dv_shared_corners: the distinct grid corners of n leaves (corner c =
 * (c & 1, c >> 1 & 1, c >> 2 & 1) of leaf (l, i, j, k) lies at finest-level grid
 * point ((i + c_x) 2^(L-l), (j + c_y) 2^(L-l), (k + c_z) 2^(L-l)), L =
 * max_level): grid[n_corners] (device, capacity 8n) receives the distinct
 * points packed as z << 42 | y << 21 | x in increasing order, index[n][8]
 * (device) every leaf corner's position in grid.  Leaves that touch the same
 * grid point share it.  DV_ERR_INVALID_ARG for a leaf level above max_level or
 * max_level > 18.
 */
dv_status dv_shared_corners(dv_ctx* ctx, const uint64_t* keys, int64_t n, int32_t max_level, uint64_t* grid,
                            uint32_t* index, int64_t* n_corners, void* stream);

/*
 * Eq. 1 soft density prior for every shared corner (grid from
 * dv_shared_corners, octree frame given by center[3] (host) and root_size):
 * dens = v_far + (v_close - v_far) exp(-2 d^2 / s_min^2), d the distance from
 * the corner to the nearest point of cloud[n_points][3] (device, world frame;
 * the paper's values are v_close = -2, v_far = -10).  Points farther than
 * 3 s_min are not searched: they would change the prior by at most
 * 8 exp(-18) ~ 1e-7, below float resolution at v_far.
 */
dv_status dv_soft_prior(dv_ctx* ctx, const uint64_t* grid, int64_t n_corners, const double* center, double root_size,
                        int32_t max_level, const float* cloud, int64_t n_points, float s_min, float v_close,
                        float v_far, float* dens, void* stream);

/*
 * One round of proximity subdivision (Sec. 3.3, step 2): every leaf whose box
 * lies within `threshold` (Euclidean point-to-box distance) of a point of cloud
 * is replaced by its eight children.  out (device, capacity 8n) receives the
 * kept leaves in input order, then child 0 of every split leaf (in input
 * order), then child 1, ..., child 7; *n_out (host) its length.  Children must
 * stay within level 18 (max_level < 18).
 */
dv_status dv_subdivide_round(dv_ctx* ctx, const uint64_t* keys, int64_t n, int32_t max_level, const double* center,
                             double root_size, const float* cloud, int64_t n_points, float threshold, uint64_t* out,
                             int64_t* n_out, void* stream);

/*
 * Visibility and height pruning of an initial grid (Sec. 3.3, step 1): keeps
 * the leaves whose box top reaches z_min (world z) and that some camera of
 * cams[n_cam] (host) sees: its 8 corners are not all in front of the near or
 * all beyond the far plane, and either the box straddles the near plane or
 * the bounding rectangle of its projected corners overlaps the image.  out
 * (device, capacity n) receives the kept keys in input order, *n_out (host)
 * their count.  Synchronises the stream.
 */
dv_status dv_visibility_prune(dv_ctx* ctx, const uint64_t* keys, int64_t n, int32_t max_level, const double* center,
                              double root_size, const dv_camera* cams, int32_t n_cam, double z_min, uint64_t* out,
                              int64_t* n_out, void* stream);

/* Per-leaf densities [n][8] from shared corner values (dens[v][c] = corner[index[v][c]]), and the
 * transpose for gradients: ADDS d_dens[v][c] into d_corner[index[v][c]] (atomics). */
dv_status dv_corner_gather(dv_ctx* ctx, const uint32_t* index, int64_t n, const float* corner, float* dens,
                           void* stream);
dv_status dv_corner_scatter(dv_ctx* ctx, const uint32_t* index, int64_t n, const float* d_dens, float* d_corner,
                            void* stream);

/*
 * Sky composite (Sec. 3.2 "Sky Modeling", Eq. 2): out = rgb + (1 - alpha) *
 * C_sky(d) per pixel, d the unit world direction of the pixel's ray, C_sky a
 * bilinear lookup of an equirectangular environment map of the world frame
 * (z up): column coordinate (atan2(d_y, d_x) + pi) / (2 pi) * env_w, row
 * coordinate acos(d_z) / pi * env_h, texel values at texel centres, wrap-around
 * in longitude, clamp to the first / last row in latitude.
 *   cams[n_cam]   host array (only intrinsics and cam_to_world.R are used)
 *   env           device [env_h][env_w][3]
 *   rgb, alpha    device inputs as written by dv_render (concatenated per camera)
 *   out           device output [sum H*W][3]; must not alias rgb when the render's
 *                 saved state is still to be differentiated (its backward reads rgb)
 * Errors: DV_ERR_INVALID_ARG / DV_ERR_INVALID_POSE / DV_ERR_CAPACITY before any
 * work is enqueued.
 */
dv_status dv_sky_composite(dv_ctx* ctx, const dv_camera* cams, int32_t n_cam, const float* env, int32_t env_h,
                           int32_t env_w, const float* rgb, const float* alpha, float* out, void* stream);

/*
 * Backward of dv_sky_composite for dL/d out (device [sum H*W][3]): ADDS
 * dL/d env into d_env ([env_h][env_w][3], atomics; NULL = skip) and ADDS
 * -dL/d out . C_sky into d_alpha ([sum H*W]; NULL = skip) -- pass that d_alpha,
 * together with dL/d rgb = dL/d out, on to dv_render_backward.
 */
dv_status dv_sky_backward(dv_ctx* ctx, const dv_camera* cams, int32_t n_cam, const float* env, int32_t env_h,
                          int32_t env_w, const float* alpha, const float* d_out, float* d_env, float* d_alpha,
                          void* stream);

/* Sizes of a saved state: visible voxels, (tile, voxel) pairs and tiles of view
 * `view`, or of the whole call for view = -1 (per-view figures synchronise the
 * state's stream).  Returns DV_ERR_INVALID_ARG for a bad index. */
dv_status dv_state_stats(const dv_state* state, int32_t view, int64_t* n_visible, int64_t* n_pairs,
                         int64_t* n_tiles);

/* Work done by the forward compositing of a saved state, over all its views
 * (`view` must be -1, or 0 for a single-view state): voxel slab tests (pixel x
 * list entry examined), actor clip-box tests, and composited segments.
 * Synchronises the state's stream.  These are the algorithmic units behind the
 * compositing roofline. */
dv_status dv_state_work(const dv_state* state, int32_t view, uint64_t* tests, uint64_t* box_tests,
                        uint64_t* segments);

/* FP32 FMA rate of device `device` (a measurement utility, no counterpart in
 * the paper): launches a kernel of independent dependent-FMA chains on every SM
 * `reps` times (after one warm-up launch), each thread running 8 x 16 x
 * `iters` FMAs, and returns the FP32 operations counted (FMA = 2) and the
 * milliseconds between CUDA events around the timed launches.  Synchronous.
 * The compositing kernels' ALU roofline divides by flops / ms. */
dv_status dv_measure_fp32_fma(int32_t device, int32_t iters, int32_t reps, double* flops, double* ms);

/* Number of kernel launches this library has issued in this process (all
 * contexts); reset to zero when `reset` is non-zero (returns the old value). */
long long dv_launch_count(int32_t reset);

/*
 * dv_render_backward without any device allocation (the paper has no
 * counterpart; this exists for callers that may not allocate while the
 * backward runs: inside a CUDA-graph capture that must hold no allocation
 * nodes, in a real-time loop that may not take an allocator lock, or with the
 * device memory fully committed to another allocator).  Same arguments,
 * results and accumulation semantics as dv_render_backward.  Its scratch is a
 * file-scope device array sized for 131072 visible voxels per render call,
 * summed over its views (6 MiB, held by every GPU that loads the library until
 * exit); a larger state fails with DV_ERR_CAPACITY before any work is enqueued.
 * All calls on a device share that array and clear the part they use first:
 * calls whose GPU work overlaps (unordered streams) race on it.  The first call
 * on a device looks up the array's address; make it before any stream capture.
 * That address is kept per device ordinal for the life of the process: a
 * caller that resets a device (cudaDeviceReset) must not use this entry point
 * on that device afterwards.
 */
dv_status dv_render_backward_static(dv_ctx* ctx, dv_state* state, const float* d_rgb, const float* d_depth,
                                    const float* d_alpha, float* const* d_dens, float* const* d_sh, void* stream);

/* Per-stage timing with CUDA events recorded on the call's stream.  While
 * enabled, every stage below is bracketed by events; dv_profile_read()
 * synchronises those events and returns, for stage k in names order, the
 * summed milliseconds and the number of times the stage ran, then resets the
 * counters.  Stages: "project", "scan", "compact", "sort_vox", "records",
 * "emit", "sort_pairs", "ranges", "composite_fwd", "composite_bwd", "sh_bwd". */
dv_status dv_profile_enable(dv_ctx* ctx, int32_t on);
/* The same for a subset of the stages: bit k of `mask` brackets stage k (names
 * order above); 0 turns profiling off.  Fewer events, less overhead in the
 * timed stream. */
dv_status dv_profile_enable_stages(dv_ctx* ctx, uint32_t mask);
dv_status dv_profile_read(dv_ctx* ctx, const char* const* names, int32_t n, double* ms, int64_t* launches);

/* ------------------------------------------------------------------------
 * Serving loop: continuous batching of render requests (no counterpart in the
 * paper; it keeps the scene resident and renders requests as they arrive).
 *
 * A request is a camera plus the pose of every octree at the request's
 * timestamp, with caller-owned device output buffers (rgb [H*W][3], depth and
 * alpha [H*W]) that must stay valid until the request is done.  Worker threads,
 * each with its own CUDA stream, take the queued requests in arrival order up
 * to the admission limits below and render each group as one batch of views
 * (dv_render_views); requests arriving meanwhile join the next batch a worker
 * forms, and the batches of different workers overlap on the GPU.  Results are
 * identical to rendering each request alone.
 *
 * Admission by device memory: each request is charged the device memory its
 * render takes from the worker's pool (the model behind dv_workspace_need: the
 * per-voxel projection arrays, per-pixel and per-tile state, and the records,
 * pairs and sort scratch of its visible voxels), with the visible fraction of
 * the scene's voxels and the pairs per tile taken from the batches already
 * rendered (conservative values before the first), plus 25%.  A request joins
 * a batch only while the charges of everything in flight stay within
 * max_inflight_bytes (a request above the budget on its own runs alone).
 * ------------------------------------------------------------------------ */
typedef struct dv_server dv_server;

typedef struct {
    int32_t max_views;           /* requests per batch, 1..DV_MAX_VIEWS (1 = one request per launch) */
    int32_t n_workers;           /* batches in flight at once, each on its own stream, 1..8 */
    int64_t max_batch_pixels;    /* pixels per batch (a larger single request still runs, alone) */
    int64_t max_inflight_pixels; /* pixels rendering at once over all workers */
    dv_opts opts;
    int64_t max_inflight_bytes;  /* device memory charged to the requests in flight, over all workers
                                    (0: no byte limit) */
} dv_serve_config;

/* Starts a server on `device` over the octrees oct[n_oct] (device buffers
 * borrowed for the server's lifetime; the dv_octree structs are copied). */
dv_status dv_serve_create(dv_server** srv, int32_t device, const dv_octree* oct, int32_t n_oct,
                          const dv_serve_config* cfg);
/* Queues one request (poses: host array [n_oct], copied); returns its ticket. */
dv_status dv_serve_submit(dv_server* srv, const dv_camera* cam, const dv_pose* poses, float* rgb, float* depth,
                          float* alpha, int64_t* ticket);
/* Non-blocking: *done = 1 once the outputs are written; then *latency_ms is the
 * time from submit to completion and the return value the request's status. */
dv_status dv_serve_poll(dv_server* srv, int64_t ticket, int32_t* done, double* latency_ms);
/* Waits at most timeout_ms for the request; DV_ERR_TIMEOUT if it is not done. */
dv_status dv_serve_wait(dv_server* srv, int64_t ticket, double timeout_ms, double* latency_ms);
/* Forgets a finished request (its ticket becomes invalid). */
dv_status dv_serve_release(dv_server* srv, int64_t ticket);
/* Batches run, requests rendered, largest batch so far. */
dv_status dv_serve_stats(dv_server* srv, int64_t* batches, int64_t* views, int64_t* max_batch);
/* Device memory charged to the requests in flight now, the largest such total
 * since the server started or the last reset, and the charge of the last
 * request admitted (bytes).  reset_peak != 0 restarts the peak from now. */
dv_status dv_serve_memory(dv_server* srv, int32_t reset_peak, int64_t* inflight_bytes, int64_t* peak_inflight_bytes,
                          int64_t* last_request_bytes);
/* Holds (paused != 0) or resumes admission: queued requests wait while paused
 * (dv_serve_destroy still finishes them). */
dv_status dv_serve_pause(dv_server* srv, int32_t paused);
const char* dv_serve_last_error(const dv_server* srv);
/* Finishes every queued request, stops the workers and frees the server. */
void dv_serve_destroy(dv_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* DV_H */
