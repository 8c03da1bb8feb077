// LiDAR-guided initialisation of the background octree (Sec. 3.3): shared grid corners, the
// soft density prior of Eq. 1 and one round of proximity subdivision.
//
//  * Shared corners: every leaf emits its 8 corner grid points (finest-level integer
//    coordinates, packed 21 bits per axis) tagged with (leaf, corner); one radix sort groups
//    equal points, a scan numbers the distinct ones, and every (leaf, corner) gets its index.
//  * Eq. 1: the LiDAR points are bucketed in a uniform grid of cell h = 3 s (sorted by cell
//    key); each corner scans the 27 cells around it for its nearest point.  A point farther
//    than 3 s changes the prior by at most 8 exp(-18) ~ 1e-7, below float32 resolution at
//    v_far, so beyond that radius the corner takes v_far.
//  * Subdivision: every LiDAR point visits, for each level, the leaf cells whose box lies within
//    the threshold of it (exact point-box distance) and looks each up in the sorted leaf keys;
//    found leaves are flagged.  The output keeps the unflagged leaves in input order, then the
//    children of the flagged ones, child 0 of every flagged leaf first, then child 1, ...
#include <cuda_runtime.h>
#include <stdint.h>

#include "dv_internal.cuh"

namespace dv {

namespace {

constexpr uint64_t kIMask = (1ull << 19) - 1;
constexpr int kCellBits = 21;
constexpr int64_t kCellOff = 1ll << (kCellBits - 1);

__device__ __forceinline__ uint64_t pack_grid(uint64_t x, uint64_t y, uint64_t z) {
    return (z << 42) | (y << 21) | x;
}

__global__ void k_corner_emit(const uint64_t* __restrict__ keys, int64_t n, int max_level, uint64_t* __restrict__ ck,
                              uint32_t* __restrict__ cv) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    const int64_t v = t >> 3;
    const int c = (int)(t & 7);
    const uint64_t k = keys[v];
    const int lev = (int)((k >> 57) & 31);
    const int sh = max_level > lev ? max_level - lev : 0;  // a level above max_level is rejected by the caller
    const uint64_t i = ((k & kIMask) + (c & 1)) << sh;
    const uint64_t j = (((k >> 19) & kIMask) + ((c >> 1) & 1)) << sh;
    const uint64_t kk = (((k >> 38) & kIMask) + ((c >> 2) & 1)) << sh;
    ck[t] = pack_grid(i, j, kk);
    cv[t] = (uint32_t)t;
}

__global__ void k_corner_flag(const uint64_t* __restrict__ sk, int64_t m, uint32_t* __restrict__ first) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    first[t] = (t == 0 || sk[t] != sk[t - 1]) ? 1u : 0u;
}

// pos = exclusive scan of first: sorted entry t belongs to distinct point pos[t] + first[t] - 1
__global__ void k_corner_assign(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                                const uint32_t* __restrict__ first, const uint32_t* __restrict__ pos, int64_t m,
                                uint64_t* __restrict__ grid_out, uint32_t* __restrict__ index_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const uint32_t id = pos[t] + first[t] - 1u;
    index_out[sv[t]] = id;
    if (first[t]) grid_out[id] = sk[t];
}

__device__ __forceinline__ uint64_t cell_key(int64_t cx, int64_t cy, int64_t cz) {
    auto cl = [](int64_t a) {
        a += kCellOff;
        return (uint64_t)(a < 0 ? 0 : (a >= (1ll << kCellBits) ? (1ll << kCellBits) - 1 : a));
    };
    return (cl(cz) << (2 * kCellBits)) | (cl(cy) << kCellBits) | cl(cx);
}

struct Frame {
    double root_min[3];
    double unit;  // finest grid step (root / 2^max_level)
};

__global__ void k_cloud_cells(const float* __restrict__ cloud, int64_t m, Frame f, double h,
                              uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int64_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = (int64_t)floor(((double)cloud[t * 3 + a] - f.root_min[a]) / h);
    key[t] = cell_key(c[0], c[1], c[2]);
    val[t] = (uint32_t)t;
}

__device__ __forceinline__ int64_t lower_bound(const uint64_t* a, int64_t n, uint64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_soft_prior(const uint64_t* __restrict__ grid, int64_t n_corners, Frame f, double h,
                             const uint64_t* __restrict__ ckey, const uint32_t* __restrict__ cidx, int64_t m,
                             const float* __restrict__ cloud, float s, float v_close, float v_far,
                             float* __restrict__ dens) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_corners) return;
    const uint64_t g = grid[t];
    double q[3];
    q[0] = f.root_min[0] + (double)(g & ((1ull << 21) - 1)) * f.unit;
    q[1] = f.root_min[1] + (double)((g >> 21) & ((1ull << 21) - 1)) * f.unit;
    q[2] = f.root_min[2] + (double)((g >> 42) & ((1ull << 21) - 1)) * f.unit;
    int64_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = (int64_t)floor((q[a] - f.root_min[a]) / h);
    // x is the key's low field, so the three cells x-1..x+1 of one (y, z) row are one run of keys:
    // one search per row.  The centre row goes first; another row is skipped when its box is
    // no nearer than the best point so far, so the minimum is still the one over all 27 cells.
    // The row's lower bound takes a slack of 1e-9 h off each axis gap: a point's cell comes from
    // a quotient below 2^21 in FP64, so it can sit at most ~5e-10 h across a cell boundary.
    double gap_lo[3], gap_hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double lo = f.root_min[a] + (double)c[a] * h;
        gap_lo[a] = fmax(0.0, q[a] - lo - 1e-9 * h);
        gap_hi[a] = fmax(0.0, lo + h - q[a] - 1e-9 * h);
    }
    double best = INFINITY;
    for (int it = 0; it < 9; ++it) {
        const int r = (it + 4) % 9;  // it = 0: the centre row
        const int dy = r % 3 - 1, dz = r / 3 - 1;
        {
            const double gy = dy < 0 ? gap_lo[1] : (dy > 0 ? gap_hi[1] : 0.0);
            const double gz = dz < 0 ? gap_lo[2] : (dz > 0 ? gap_hi[2] : 0.0);
            if (gy * gy + gz * gz >= best) continue;
        }
        {
            const uint64_t k_lo = cell_key(c[0] - 1, c[1] + dy, c[2] + dz);
            const uint64_t k_hi = cell_key(c[0] + 1, c[1] + dy, c[2] + dz);
            for (int64_t e = lower_bound(ckey, m, k_lo); e < m && ckey[e] <= k_hi; ++e) {
                const uint32_t p = cidx[e];
                const double ex = (double)cloud[p * 3 + 0] - q[0], ey = (double)cloud[p * 3 + 1] - q[1],
                             ez = (double)cloud[p * 3 + 2] - q[2];
                best = fmin(best, ex * ex + ey * ey + ez * ez);
            }
        }
    }
    // Eq. 1 (beyond the 27-cell radius the exponential is below float resolution at v_far)
    const double ss = (double)s * (double)s;
    const double e = best < INFINITY ? exp(-2.0 * best / ss) : 0.0;
    dens[t] = (float)((double)v_far + ((double)v_close - (double)v_far) * e);
}

// one thread per LiDAR point: flag the leaves (sorted keys) whose box lies within thr of it
__global__ void k_subdiv_flags(const float* __restrict__ cloud, int64_t m, Frame f, double root_size, uint32_t levels,
                               double thr, const uint64_t* __restrict__ skeys, const uint32_t* __restrict__ sidx,
                               int64_t n, uint8_t* __restrict__ split) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    double p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = (double)cloud[t * 3 + a] - f.root_min[a];
    for (int l = 0; l < 32; ++l) {
        if (!((levels >> l) & 1u)) continue;  // only levels that hold leaves
        const double s = ldexp(root_size, -l);
        const int64_t lim = (1ll << l) - 1;
        int64_t lo[3], hi[3];
        bool any = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int64_t)floor((p[a] - thr) / s);
            hi[a] = (int64_t)floor((p[a] + thr) / s);
            lo[a] = lo[a] < 0 ? 0 : lo[a];
            hi[a] = hi[a] > lim ? lim : hi[a];
            any = any && lo[a] <= hi[a];
        }
        if (!any) continue;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    const int64_t ij[3] = {x, y, z};
                    double d2 = 0.0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const double b0 = (double)ij[a] * s, b1 = b0 + s;
                        const double g = fmax(fmax(b0 - p[a], 0.0), p[a] - b1);
                        d2 += g * g;
                    }
                    if (d2 > thr * thr) continue;
                    const uint64_t key = ((uint64_t)l << 57) | ((uint64_t)z << 38) | ((uint64_t)y << 19) | (uint64_t)x;
                    const int64_t e = lower_bound(skeys, n, key);
                    if (e < n && skeys[e] == key) split[sidx[e]] = 1;
                }
    }
}

__global__ void k_subdiv_write(const uint64_t* __restrict__ keys, int64_t n, const uint8_t* __restrict__ split,
                               const uint32_t* __restrict__ pos_keep, const uint32_t* __restrict__ pos_split,
                               int64_t n_keep, int64_t n_split, uint64_t* __restrict__ out) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint64_t k = keys[v];
    if (!split[v]) {
        out[pos_keep[v]] = k;
        return;
    }
    const uint64_t lev = (k >> 57) & 31, i = k & kIMask, j = (k >> 19) & kIMask, kk = (k >> 38) & kIMask;
    for (int c = 0; c < 8; ++c)
        out[n_keep + (int64_t)c * n_split + pos_split[v]] =
            ((lev + 1) << 57) | ((2 * kk + ((c >> 2) & 1)) << 38) | ((2 * j + ((c >> 1) & 1)) << 19) |
            (2 * i + (c & 1));
}

__global__ void k_not(const uint8_t* __restrict__ a, int64_t n, uint32_t* __restrict__ yes, uint32_t* __restrict__ no) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    yes[t] = a[t] ? 1u : 0u;
    no[t] = a[t] ? 0u : 1u;
}

// v[t] = t, and the set of leaf levels present (bit l of *levels)
__global__ void k_iota_levels(const uint64_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ v,
                              uint32_t* __restrict__ levels) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    v[t] = (uint32_t)t;
    atomicOr(levels, 1u << ((keys[t] >> 57) & 31));
}

unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// per-leaf densities [n][8] from shared corner values, and the transpose for gradients
__global__ void k_corner_gather(const uint32_t* __restrict__ index, int64_t n8, const float* __restrict__ corner,
                                float* __restrict__ dens) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n8) return;
    dens[t] = corner[index[t]];
}

__global__ void k_corner_scatter(const uint32_t* __restrict__ index, int64_t n8, const float* __restrict__ d_dens,
                                 float* __restrict__ d_corner) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n8) return;
    const float g = d_dens[t];
    if (g != 0.0f) atomicAdd(d_corner + index[t], g);
}

// level of every key (bit mask) to validate against max_level
__global__ void k_levels(const uint64_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ levels) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    atomicOr(levels, 1u << ((keys[t] >> 57) & 31));
}

// a leaf is kept if its box top reaches z_min and some camera sees it (see the header)
__global__ void k_visible(const uint64_t* __restrict__ keys, int64_t n, Frame f, double root_size,
                          const InitCam* __restrict__ cams, int n_cam, double z_min, uint32_t* __restrict__ keep) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint64_t k = keys[v];
    const int lev = (int)((k >> 57) & 31);
    const double s = ldexp(root_size, -lev);
    const double lo[3] = {f.root_min[0] + (double)(k & kIMask) * s, f.root_min[1] + (double)((k >> 19) & kIMask) * s,
                          f.root_min[2] + (double)((k >> 38) & kIMask) * s};
    uint32_t vis = 0;
    if (lo[2] + s >= z_min) {
        for (int c = 0; c < n_cam && !vis; ++c) {
            const InitCam& C = cams[c];
            int behind = 0, beyond = 0;
            double u0 = INFINITY, u1 = -INFINITY, w0 = INFINITY, w1 = -INFINITY;
            for (int q = 0; q < 8; ++q) {
                const double p[3] = {lo[0] + ((q & 1) ? s : 0.0) - C.t[0], lo[1] + ((q & 2) ? s : 0.0) - C.t[1],
                                     lo[2] + ((q & 4) ? s : 0.0) - C.t[2]};
                // camera frame: R^T (p - t), R row-major camera -> world
                const double x = C.R[0] * p[0] + C.R[3] * p[1] + C.R[6] * p[2];
                const double y = C.R[1] * p[0] + C.R[4] * p[1] + C.R[7] * p[2];
                const double z = C.R[2] * p[0] + C.R[5] * p[1] + C.R[8] * p[2];
                behind += z < C.near_;
                beyond += z > C.far_;
                if (z >= C.near_) {
                    const double u = C.fx * x / z + C.cx, w = C.fy * y / z + C.cy;
                    u0 = fmin(u0, u);
                    u1 = fmax(u1, u);
                    w0 = fmin(w0, w);
                    w1 = fmax(w1, w);
                }
            }
            if (behind == 8 || beyond == 8) continue;
            if (behind > 0)
                vis = 1;
            else
                vis = (u1 >= 0.0 && u0 <= (double)C.W && w1 >= 0.0 && w0 <= (double)C.H) ? 1u : 0u;
        }
    }
    keep[v] = vis;
}

__global__ void k_compact_keys(const uint64_t* __restrict__ keys, int64_t n, const uint32_t* __restrict__ keep,
                               const uint32_t* __restrict__ pos, uint64_t* __restrict__ out) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || !keep[v]) return;
    out[pos[v]] = keys[v];
}

}  // namespace

static Frame make_frame(const double* center, double root_size, int max_level);

cudaError_t visibility_prune(const uint64_t* keys, int64_t n, const double* center, double root_size,
                             const InitCam* cams_host, int n_cam, double z_min, uint64_t* out, int64_t* n_out,
                             Arena& ar, cudaStream_t s) {
    *n_out = 0;
    if (n <= 0) return cudaSuccess;
    const Frame f = make_frame(center, root_size, 0);
    InitCam* cams = ar.alloc<InitCam>((size_t)(n_cam > 0 ? n_cam : 1));
    uint32_t* keep = ar.alloc<uint32_t>(n);
    uint32_t* pos = ar.alloc<uint32_t>(n);
    uint32_t* tot = ar.alloc<uint32_t>(1);
    if (ar.err != cudaSuccess) return ar.err;
    cudaError_t e = cudaSuccess;
    if (n_cam > 0) e = cudaMemcpyAsync(cams, cams_host, sizeof(InitCam) * n_cam, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_visible<<<nb(n), 256, 0, s>>>(keys, n, f, root_size, cams, n_cam, z_min, keep);
    count_launches(1);
    e = scan_u32_to_u32(keep, pos, n, tot, ar, s);
    if (e != cudaSuccess) return e;
    k_compact_keys<<<nb(n), 256, 0, s>>>(keys, n, keep, pos, out);
    count_launches(1);
    uint32_t h = 0;
    e = cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *n_out = h;
    return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t corner_gather(const uint32_t* index, int64_t n, const float* corner, float* dens, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_corner_gather<<<nb(n * 8), 256, 0, s>>>(index, n * 8, corner, dens);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t corner_scatter(const uint32_t* index, int64_t n, const float* d_dens, float* d_corner, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_corner_scatter<<<nb(n * 8), 256, 0, s>>>(index, n * 8, d_dens, d_corner);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t key_levels(const uint64_t* keys, int64_t n, uint32_t* levels_host, Arena& ar, cudaStream_t s) {
    *levels_host = 0;
    if (n <= 0) return cudaSuccess;
    uint32_t* d = ar.alloc<uint32_t>(1);
    if (!d) return ar.err;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_levels<<<nb(n), 256, 0, s>>>(keys, n, d);
    count_launches(1);
    e = cudaMemcpyAsync(levels_host, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

cudaError_t shared_corners(const uint64_t* keys, int64_t n, int max_level, uint64_t* grid_out, uint32_t* index_out,
                           int64_t* n_corners, Arena& ar, cudaStream_t s, bool* sort_timeout) {
    *n_corners = 0;
    *sort_timeout = false;
    if (n <= 0) return cudaSuccess;
    const int64_t m = n * 8;
    uint64_t* k0 = ar.alloc<uint64_t>(m);
    uint64_t* k1 = ar.alloc<uint64_t>(m);
    uint32_t* v0 = ar.alloc<uint32_t>(m);
    uint32_t* v1 = ar.alloc<uint32_t>(m);
    uint32_t* first = ar.alloc<uint32_t>(m);
    uint32_t* pos = ar.alloc<uint32_t>(m);
    uint32_t* total = ar.alloc<uint32_t>(2);  // [0] distinct corners, [1] the sort's wait flag
    if (ar.err != cudaSuccess) return ar.err;
    cudaError_t e = cudaMemsetAsync(total + 1, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_corner_emit<<<nb(m), 256, 0, s>>>(keys, n, max_level, k0, v0);
    count_launches(1);
    uint64_t* kk = k0;
    uint32_t* vv = v0;
    e = radix_sort_u64(kk, vv, k1, v1, m, 63, ar, s, total + 1);
    if (e != cudaSuccess) return e;
    k_corner_flag<<<nb(m), 256, 0, s>>>(kk, m, first);
    count_launches(1);
    e = scan_u32_to_u32(first, pos, m, total, ar, s);
    if (e != cudaSuccess) return e;
    k_corner_assign<<<nb(m), 256, 0, s>>>(kk, vv, first, pos, m, grid_out, index_out);
    count_launches(1);
    uint32_t h[2] = {0, 0};
    e = cudaMemcpyAsync(h, total, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *n_corners = h[0];
    *sort_timeout = h[1] != 0;
    return e == cudaSuccess ? cudaGetLastError() : e;
}

static Frame make_frame(const double* center, double root_size, int max_level) {
    Frame f;
    for (int a = 0; a < 3; ++a) f.root_min[a] = center[a] - 0.5 * root_size;
    f.unit = ldexp(root_size, -max_level);
    return f;
}

cudaError_t soft_prior(const uint64_t* grid, int64_t n_corners, const double* center, double root_size, int max_level,
                       const float* cloud, int64_t m, float s_min, float v_close, float v_far, float* dens, Arena& ar,
                       cudaStream_t s, bool* sort_timeout) {
    *sort_timeout = false;
    if (n_corners <= 0) return cudaSuccess;
    const Frame f = make_frame(center, root_size, max_level);
    const double h = 3.0 * (double)s_min;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr;
    uint32_t* flag = nullptr;
    if (m > 0) {
        k0 = ar.alloc<uint64_t>(m);
        k1 = ar.alloc<uint64_t>(m);
        v0 = ar.alloc<uint32_t>(m);
        v1 = ar.alloc<uint32_t>(m);
        flag = ar.alloc<uint32_t>(1);
        if (ar.err != cudaSuccess) return ar.err;
        cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        k_cloud_cells<<<nb(m), 256, 0, s>>>(cloud, m, f, h, k0, v0);
        count_launches(1);
        e = radix_sort_u64(k0, v0, k1, v1, m, 3 * kCellBits, ar, s, flag);
        if (e != cudaSuccess) return e;
    }
    k_soft_prior<<<nb(n_corners), 256, 0, s>>>(grid, n_corners, f, h, k0, v0, m, cloud, s_min, v_close, v_far, dens);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (flag) {
        // the cell sort's own wait flag: a run-out look-back left the cloud unsorted (wrong nearest points)
        uint32_t hf = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flag, sizeof(hf), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *sort_timeout = hf != 0;
    }
    return e;
}

cudaError_t subdivide_round(const uint64_t* keys, int64_t n, const double* center, double root_size, int max_level,
                            const float* cloud, int64_t m, float thr, uint64_t* out, int64_t* n_out, Arena& ar,
                            cudaStream_t s, bool* sort_timeout) {
    *n_out = n;
    *sort_timeout = false;
    if (n <= 0) return cudaSuccess;
    const Frame f = make_frame(center, root_size, max_level);
    uint64_t* k0 = ar.alloc<uint64_t>(n);
    uint64_t* k1 = ar.alloc<uint64_t>(n);
    uint32_t* v0 = ar.alloc<uint32_t>(n);
    uint32_t* v1 = ar.alloc<uint32_t>(n);
    uint8_t* split = ar.alloc<uint8_t>(n);
    uint32_t* yes = ar.alloc<uint32_t>(n);
    uint32_t* no = ar.alloc<uint32_t>(n);
    uint32_t* pos_s = ar.alloc<uint32_t>(n);
    uint32_t* pos_k = ar.alloc<uint32_t>(n);
    uint32_t* tot = ar.alloc<uint32_t>(2);
    uint32_t* lvl = ar.alloc<uint32_t>(2);  // [0] levels present, [1] the sort's wait flag
    if (ar.err != cudaSuccess) return ar.err;
    cudaError_t e = cudaMemcpyAsync(k0, keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(split, 0, n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(lvl, 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_iota_levels<<<nb(n), 256, 0, s>>>(keys, n, v0, lvl);
    count_launches(1);
    uint64_t* kk = k0;
    uint32_t* vv = v0;
    e = radix_sort_u64(kk, vv, k1, v1, n, 62, ar, s, lvl + 1);
    if (e != cudaSuccess) return e;
    uint32_t lv[2] = {0, 0};
    e = cudaMemcpyAsync(lv, lvl, sizeof(lv), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const uint32_t levels = lv[0];
    if (lv[1]) {
        // the key sort's bounded wait ran out: its order is wrong, so no leaf lookup is trusted
        *sort_timeout = true;
        return cudaSuccess;
    }
    if (m > 0) {
        k_subdiv_flags<<<nb(m), 256, 0, s>>>(cloud, m, f, root_size, levels, thr, kk, vv, n, split);
        count_launches(1);
    }
    k_not<<<nb(n), 256, 0, s>>>(split, n, yes, no);
    count_launches(1);
    e = scan_u32_to_u32(yes, pos_s, n, tot, ar, s);
    if (e == cudaSuccess) e = scan_u32_to_u32(no, pos_k, n, tot + 1, ar, s);
    uint32_t h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const int64_t n_split = h[0], n_keep = h[1];
    k_subdiv_write<<<nb(n), 256, 0, s>>>(keys, n, split, pos_k, pos_s, n_keep, n_split, out);
    count_launches(1);
    *n_out = n_keep + 8 * n_split;
    return cudaGetLastError();
}

}  // namespace dv

namespace dv {

namespace {

// leaf t of the uniform grid: (i, j, k) = (t mod n, (t / n) mod n, t / n^2), n = 2^level
__global__ void k_asset_grid(int level, float v_init, int64_t n_leaf, uint64_t* __restrict__ keys,
                             float4* __restrict__ dens) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_leaf) return;
    const uint64_t n = 1ull << level;
    const uint64_t i = (uint64_t)t & (n - 1), j = ((uint64_t)t >> level) & (n - 1), k = (uint64_t)t >> (2 * level);
    keys[t] = ((uint64_t)level << 57) | (k << 38) | (j << 19) | i;
    const float4 v = make_float4(v_init, v_init, v_init, v_init);
    dens[2 * t] = v;
    dens[2 * t + 1] = v;
}

}  // namespace

cudaError_t asset_grid(int level, float v_init, uint64_t* keys, float* dens, cudaStream_t s) {
    const int64_t n = (int64_t)1 << (3 * level);
    k_asset_grid<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(level, v_init, n, keys, reinterpret_cast<float4*>(dens));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dv
