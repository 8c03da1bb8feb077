// Per-voxel projection, visibility compaction, render records and tile binning.
//
// All kernels run over every view of a render call at once (a view is one camera
// of one request, with its own actor poses); tiles are numbered globally.
//
// project  (one thread per (view, voxel) of every octree): leaf geometry from its key,
//          the 8 corners placed in the camera frame by the composed pose
//          (local -> world -> camera, Sec. 3.2), near/far culling, a conservative
//          screen rectangle of the box (clipped against the near plane) turned
//          into a tile rectangle, and the depth-order key.
// records  (one thread per visible voxel, in depth-key order): 64-byte record
//          with the local box, the 8 raw densities and the view-dependent SH
//          colour for this camera.
// emit     one (tile, record) pair per tile of the rectangle.
// ranges   [start, end) of every tile in the tile-sorted pair list.
//
// Depth-order key.  Leaves of one octree are cells of a binary space partition
// (each node split by the three planes through its centre).  For rays that all
// start at one point o (a pinhole), visiting at every node the children on o's
// side of each splitting plane first gives a front-to-back order that holds
// for every ray at once: a ray from o meets the half-space containing o before
// it crosses the plane, and never crosses back.  The key spells the leaf's
// path with each child bit flipped when o lies on the positive side of that
// node's plane, so sorting keys ascending yields that order.  The side tests
// are exact integer comparisons of 2*(o - root_min)/root*2^L against the
// node-centre lattice coordinates.  The view and octree indices sit above the
// path bits, so one sort groups each (view, octree) and orders it front to back.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dv_internal.cuh"

namespace dv {

namespace {

constexpr uint64_t M19 = (1ull << 19) - 1;

__device__ __forceinline__ int find_octree(const BatchParams& bp, int64_t g) {
    int lo = 0, hi = bp.n_oct - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (bp.vox_offset[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

struct Leaf {
    int level;
    uint32_t i, j, k;
    float mn[3];
    float s;
};

__device__ __forceinline__ Leaf decode_leaf(const OctParams& P, uint64_t key) {
    Leaf L;
    L.level = (int)((key >> 57) & 31ull);
    L.i = (uint32_t)(key & M19);
    L.j = (uint32_t)((key >> 19) & M19);
    L.k = (uint32_t)((key >> 38) & M19);
    L.s = ldexpf(P.root_size, -L.level);
    L.mn[0] = fmaf((float)L.i, L.s, P.root_min[0]);
    L.mn[1] = fmaf((float)L.j, L.s, P.root_min[1]);
    L.mn[2] = fmaf((float)L.k, L.s, P.root_min[2]);
    return L;
}

__device__ __forceinline__ void proj_point(const ViewParams& fp, float x, float y, float z, float& u0, float& u1,
                                           float& v0, float& v1) {
    float iz = 1.0f / z;
    float u = fmaf(fp.fx * x, iz, fp.cx);
    float v = fmaf(fp.fy * y, iz, fp.cy);
    u0 = fminf(u0, u);
    u1 = fmaxf(u1, u);
    v0 = fminf(v0, v);
    v1 = fmaxf(v1, v);
}

// Projection of (view, voxel) g; sets cnt[g], vis[g] (and rect[g], skey[g] when visible)
// and returns the tile count (0: not visible).
__device__ __forceinline__ uint32_t project_voxel(const BatchParams& bp, int64_t g, uint32_t* __restrict__ cnt,
                                                  uint64_t* __restrict__ rect, uint64_t* __restrict__ skey,
                                                  uint32_t* __restrict__ vis, uint32_t* __restrict__ flags) {
    const int view = (int)(g / bp.n_vox);
    const int64_t gv = g - (int64_t)view * bp.n_vox;
    const int o = find_octree(bp, gv);
    const ViewParams& fp = bp.views[view];
    const OctParams& P = bp.octs[view * bp.n_oct + o];
    const int64_t v = gv - bp.vox_offset[o];
    const uint64_t key = P.key[v];
    cnt[g] = 0;
    vis[g] = 0;
    const Leaf L = decode_leaf(P, key);
    if (L.level > P.max_level || L.i >> L.level || L.j >> L.level || L.k >> L.level) {
        atomicOr(flags, DV_FLAG_BAD_LEVEL);
        return 0;
    }
    // corners in the camera frame: p = M (mn + s*offset) + m
    float p0[3], e[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        p0[r] = fmaf(P.M[r * 3 + 0], L.mn[0], fmaf(P.M[r * 3 + 1], L.mn[1], fmaf(P.M[r * 3 + 2], L.mn[2], P.m[r])));
#pragma unroll
        for (int c = 0; c < 3; ++c) e[c][r] = P.M[r * 3 + c] * L.s;
    }
    float cz[8], cx[8], cy[8];
    float zmin = INFINITY, zmax = -INFINITY;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float x = p0[0], y = p0[1], z = p0[2];
        if (c & 1) x += e[0][0], y += e[0][1], z += e[0][2];
        if (c & 2) x += e[1][0], y += e[1][1], z += e[1][2];
        if (c & 4) x += e[2][0], y += e[2][1], z += e[2][2];
        cx[c] = x;
        cy[c] = y;
        cz[c] = z;
        zmin = fminf(zmin, z);
        zmax = fmaxf(zmax, z);
    }
    if (zmax < fp.z_clip || zmin > fp.far_) return 0;
    float u0 = INFINITY, u1 = -INFINITY, w0 = INFINITY, w1 = -INFINITY;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (cz[c] >= fp.z_clip) proj_point(fp, cx[c], cy[c], cz[c], u0, u1, w0, w1);
    if (zmin < fp.z_clip) {
        // edges crossing the clip plane contribute their crossing points
#pragma unroll
        for (int bit = 1; bit < 8; bit <<= 1) {
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                if (a & bit) continue;
                const int b = a | bit;
                const float za = cz[a], zb = cz[b];
                if ((za < fp.z_clip) != (zb < fp.z_clip)) {
                    const float t = (fp.z_clip - za) / (zb - za);
                    proj_point(fp, fmaf(t, cx[b] - cx[a], cx[a]), fmaf(t, cy[b] - cy[a], cy[a]), fp.z_clip, u0, u1,
                               w0, w1);
                }
            }
        }
    }
    // pixels whose centres (u+0.5, v+0.5) may fall inside the silhouette, with a rounding margin
    const float mu = 0.1f + 4e-6f * fmaxf(fabsf(u0), fabsf(u1));
    const float mv = 0.1f + 4e-6f * fmaxf(fabsf(w0), fabsf(w1));
    const float lu = fmaxf(u0 - 0.5f - mu, -1.0f), hu = fminf(u1 - 0.5f + mu, (float)fp.W + 1.0f);
    const float lv = fmaxf(w0 - 0.5f - mv, -1.0f), hv = fminf(w1 - 0.5f + mv, (float)fp.H + 1.0f);
    const int pu0 = max((int)ceilf(lu), 0), pu1 = min((int)floorf(hu), fp.W - 1);
    const int pv0 = max((int)ceilf(lv), 0), pv1 = min((int)floorf(hv), fp.H - 1);
    if (!(pu0 <= pu1 && pv0 <= pv1)) return 0;
    const uint32_t tx0 = pu0 >> 4, tx1 = pu1 >> 4, ty0 = pv0 >> 4, ty1 = pv1 >> 4;
    const uint32_t n_tiles = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    cnt[g] = n_tiles;
    vis[g] = 1;
    // pixel rectangle (tiles are its pixels >> 4)
    rect[g] = (uint64_t)pu0 | ((uint64_t)pu1 << 16) | ((uint64_t)pv0 << 32) | ((uint64_t)pv1 << 48);
    // depth-order key (see the file comment)
    uint64_t bsp = 0;
    const int Lk = bp.Lkey;
    for (int l = 0; l < L.level; ++l) {
        const int sh = L.level - 1 - l;
        const uint32_t bi = (L.i >> sh) & 1u, bj = (L.j >> sh) & 1u, bk = (L.k >> sh) & 1u;
        const int64_t ti = ((int64_t)(L.i >> (sh + 1)) * 2 + 1) << (Lk - l);
        const int64_t tj = ((int64_t)(L.j >> (sh + 1)) * 2 + 1) << (Lk - l);
        const int64_t tk = ((int64_t)(L.k >> (sh + 1)) * 2 + 1) << (Lk - l);
        const uint32_t fi = bi ^ (uint32_t)(P.O2[0] >= ti);
        const uint32_t fj = bj ^ (uint32_t)(P.O2[1] >= tj);
        const uint32_t fk = bk ^ (uint32_t)(P.O2[2] >= tk);
        bsp = (bsp << 3) | (fi << 2) | (fj << 1) | fk;
    }
    bsp <<= 3 * (Lk - L.level);
    skey[g] = ((uint64_t)view << bp.view_shift) | ((uint64_t)o << bp.oct_shift) | bsp;
    return n_tiles;
}

// One thread per (view, voxel); the block's visible voxels and (tile, voxel) pairs are
// added to totals[0] and totals[1], so the host learns both sizes from this kernel alone.
__global__ void __launch_bounds__(256) k_project(const __grid_constant__ BatchParams bp, uint32_t* __restrict__ cnt,
                                                 uint64_t* __restrict__ rect, uint64_t* __restrict__ skey,
                                                 uint32_t* __restrict__ vis, uint32_t* __restrict__ flags,
                                                 unsigned long long* __restrict__ totals) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // view * n_vox + voxel
    uint32_t c = 0;
    if (g < bp.n_vox * bp.n_view) c = project_voxel(bp, g, cnt, rect, skey, vis, flags);
    unsigned long long nv = c ? 1ull : 0ull, np = c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        nv += __shfl_down_sync(0xffffffffu, nv, off);
        np += __shfl_down_sync(0xffffffffu, np, off);
    }
    __shared__ unsigned long long s_nv[8], s_np[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_nv[warp] = nv;
        s_np[warp] = np;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            nv += s_nv[w];
            np += s_np[w];
        }
        if (nv) atomicAdd(totals + 0, nv);
        if (np) atomicAdd(totals + 1, np);
    }
}

__global__ void k_compact(const uint32_t* __restrict__ vis, const uint32_t* __restrict__ pos,
                          const uint64_t* __restrict__ skey, int64_t n, uint64_t* __restrict__ out_key,
                          uint32_t* __restrict__ out_val) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n || !vis[g]) return;
    const uint32_t p = pos[g];
    out_key[p] = skey[g];
    out_val[p] = (uint32_t)g;
}

// Real SH basis (degree <= 3) times coefficients, for a unit direction.
// Constants: 1/(2 sqrt(pi)), sqrt(3/(4 pi)), sqrt(15/(4 pi)), sqrt(5/(16 pi)),
// sqrt(15/(16 pi)), sqrt(35/(32 pi)), sqrt(105/(4 pi)), sqrt(21/(32 pi)),
// sqrt(7/(16 pi)), sqrt(105/(16 pi)); odd-m terms carry the Condon-Shortley sign.
__device__ __forceinline__ void sh_eval_basis(int deg, float x, float y, float z, float* b) {
    b[0] = 0.28209479177387814f;
    if (deg < 1) return;
    b[1] = -0.48860251190291992f * y;
    b[2] = 0.48860251190291992f * z;
    b[3] = -0.48860251190291992f * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    b[4] = 1.0925484305920792f * x * y;
    b[5] = -1.0925484305920792f * y * z;
    b[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
    b[7] = -1.0925484305920792f * x * z;
    b[8] = 0.54627421529603959f * (xx - yy);
    if (deg < 3) return;
    b[9] = -0.59004358992664352f * y * (3.0f * xx - yy);
    b[10] = 2.8906114426405538f * x * y * z;
    b[11] = -0.45704579946446572f * y * (4.0f * zz - xx - yy);
    b[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    b[13] = -0.45704579946446572f * x * (4.0f * zz - xx - yy);
    b[14] = 1.4453057213202769f * z * (xx - yy);
    b[15] = -0.59004358992664352f * x * (xx - 3.0f * yy);
}

__global__ void __launch_bounds__(256) k_records(const __grid_constant__ BatchParams bp,
                                                 const uint32_t* __restrict__ sorted_g, int64_t n_vis,
                                                 const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ rect,
                                                 VoxRec* __restrict__ rec, float4* __restrict__ nrm,
                                                 uint32_t* __restrict__ cnt_sorted,
                                                 uint64_t* __restrict__ rect_sorted) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_vis) return;
    const uint32_t g = sorted_g[r];
    const int view = (int)(g / bp.n_vox);
    const int64_t gv = (int64_t)g - (int64_t)view * bp.n_vox;
    const int o = find_octree(bp, gv);
    const OctParams& P = bp.octs[view * bp.n_oct + o];
    const int64_t v = gv - bp.vox_offset[o];
    const Leaf L = decode_leaf(P, P.key[v]);
    const float4* d4 = reinterpret_cast<const float4*>(P.dens + v * 8);
    const float4 da = __ldg(d4), db = __ldg(d4 + 1);
    // min corner relative to the camera centre (octree frame), then the view direction:
    // camera centre -> voxel centre
    const float rx = L.mn[0] - P.o_loc[0], ry = L.mn[1] - P.o_loc[1], rz = L.mn[2] - P.o_loc[2];
    float gx = fmaf(0.5f, L.s, rx);
    float gy = fmaf(0.5f, L.s, ry);
    float gz = fmaf(0.5f, L.s, rz);
    const float gl = sqrtf(gx * gx + gy * gy + gz * gz);
    const float ig = gl > 0.0f ? 1.0f / gl : 0.0f;
    gx *= ig;
    gy *= ig;
    gz *= ig;
    float b[16];
    sh_eval_basis(P.sh_degree, gx, gy, gz, b);
    const int nsh = (P.sh_degree + 1) * (P.sh_degree + 1);
    const float* shv = P.sh + v * nsh * 3;
    float cc[3] = {0.5f, 0.5f, 0.5f};
    if ((nsh * 3) % 4 == 0 && (reinterpret_cast<uintptr_t>(shv) & 15) == 0) {
        // 16-byte loads of the coefficient rows, flattened: element e = 3 q + channel
#pragma unroll
        for (int e0 = 0; e0 < 48; e0 += 4) {
            if (e0 >= nsh * 3) break;
            const float4 x4 = __ldg(reinterpret_cast<const float4*>(shv + e0));
            const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) cc[(e0 + i) % 3] = fmaf(b[(e0 + i) / 3], xs[i], cc[(e0 + i) % 3]);
        }
    } else {
        for (int q = 0; q < nsh; ++q) {
            cc[0] = fmaf(b[q], __ldg(shv + q * 3 + 0), cc[0]);
            cc[1] = fmaf(b[q], __ldg(shv + q * 3 + 1), cc[1]);
            cc[2] = fmaf(b[q], __ldg(shv + q * 3 + 2), cc[2]);
        }
    }
    const float c0 = cc[0], c1 = cc[1], c2 = cc[2];
    VoxRec R;
    R.v[0] = make_float4(rx, ry, rz, L.s);
    // the trilinear field as a polynomial in the voxel coordinates (x, y, z) in [0, 1]^3:
    // rho = c0 + c1 x + c2 y + c3 z + c4 xy + c5 xz + c6 yz + c7 xyz, from corner c = x + 2y + 4z
    const float p1 = da.y - da.x, p2 = da.z - da.x, p3 = db.x - da.x;
    const float p4 = (da.w - da.z) - p1, p5 = (db.y - db.x) - p1, p6 = (db.z - db.x) - p2;
    const float p7 = ((db.w - db.z) - (db.y - db.x)) - ((da.w - da.z) - p1);
    R.v[1] = make_float4(da.x, p1, p2, p4);
    R.v[2] = make_float4(p3, p5, p6, p7);
    R.v[3] = make_float4(fmaxf(c0, 0.0f), fmaxf(c1, 0.0f), fmaxf(c2, 0.0f), 1.0f / L.s);
    rec[r] = R;
    if (nrm) {
        // voxel normal: minus the direction of the trilinear density gradient at the voxel centre
        // (per axis: the four corners on its high side minus the four on its low side), rotated
        // into the world frame by the octree's pose
        const float gxl = (da.y + da.w + db.y + db.w) - (da.x + da.z + db.x + db.z);
        const float gyl = (da.z + da.w + db.z + db.w) - (da.x + da.y + db.x + db.y);
        const float gzl = (db.x + db.y + db.z + db.w) - (da.x + da.y + da.z + da.w);
        const float g2 = fmaf(gxl, gxl, fmaf(gyl, gyl, gzl * gzl));
        const float s = g2 > 0.0f ? -rsqrtf(g2) : 0.0f;
        const float nl[3] = {gxl * s, gyl * s, gzl * s};
        float nw[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) nw[k] = fmaf(P.Rw[k * 3 + 0], nl[0], fmaf(P.Rw[k * 3 + 1], nl[1], P.Rw[k * 3 + 2] * nl[2]));
        nrm[r] = make_float4(nw[0], nw[1], nw[2], 0.0f);
    }
    cnt_sorted[r] = cnt[g];
    rect_sorted[r] = rect[g];
}

// (view, octree) group of a depth key: view * n_oct + octree
__device__ __forceinline__ int key_group(const BatchParams& bp, uint64_t k) {
    const int view = (int)(k >> bp.view_shift);
    const int o = (int)((k >> bp.oct_shift) & ((1ull << (bp.view_shift - bp.oct_shift)) - 1));
    return view * bp.n_oct + o;
}

__global__ void k_vis_start(const __grid_constant__ BatchParams bp, const uint64_t* __restrict__ key, int64_t n_vis,
                            uint32_t* __restrict__ vis_start) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_vis) return;
    const int grp = key_group(bp, key[r]);
    const int prev = r > 0 ? key_group(bp, key[r - 1]) : -1;
    for (int q = prev + 1; q <= grp; ++q) vis_start[q] = (uint32_t)r;
    if (r == n_vis - 1)
        for (int q = grp + 1; q <= bp.n_view * bp.n_oct; ++q) vis_start[q] = (uint32_t)n_vis;
}

// one thread per (tile, voxel) pair: the pair's voxel is the last record whose first
// pair offset is <= the pair index (binary search), its tile the matching cell of
// the voxel's tile rectangle (row-major), so every thread writes exactly one pair
__global__ void k_emit(const __grid_constant__ BatchParams bp, const uint64_t* __restrict__ off,
                       const uint64_t* __restrict__ rect_sorted, const uint32_t* __restrict__ sorted_g,
                       int64_t n_vis, int64_t n_pairs, uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    int64_t lo = 0, hi = n_vis - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= (uint64_t)p)
            lo = mid;
        else
            hi = mid - 1;
    }
    const uint64_t rc = __ldg(rect_sorted + lo);
    const uint32_t tx0 = (rc & 0xffff) >> 4, tx1 = ((rc >> 16) & 0xffff) >> 4, ty0 = ((rc >> 32) & 0xffff) >> 4;
    const uint32_t w = tx1 - tx0 + 1;
    const uint32_t k = (uint32_t)((uint64_t)p - __ldg(off + lo));
    const int view = (int)(__ldg(sorted_g + lo) / (uint64_t)bp.n_vox);
    const uint32_t tiles_x = (uint32_t)bp.views[view].tiles_x;
    pkey[p] = (uint32_t)bp.tile_base[view] + (ty0 + k / w) * tiles_x + tx0 + k % w;
    pval[p] = (uint32_t)lo;
}

// For every sorted pair: which of the tile's eight 8x4-pixel blocks (bit sy*2+sx for
// the block at x in [8 sx, 8 sx + 8), y in [4 sy, 4 sy + 4)) the voxel's pixel
// rectangle touches; a warp rendering a block skips the pairs without its bit.
__device__ __forceinline__ int view_of_tile(const BatchParams& bp, int t) {
    int lo = 0, hi = bp.n_view - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bp.tile_base[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// one thread per tile-sorted pair: the 8x4-pixel blocks of its tile the voxel's pixel rectangle
// touches (bit sy * 2 + sx), and the tile's list range from the key boundaries
__global__ void k_pair_mask(const __grid_constant__ BatchParams bp, const uint32_t* __restrict__ pkey,
                            const uint32_t* __restrict__ pval, const uint64_t* __restrict__ rect_sorted,
                            int64_t n_pairs, uint8_t* __restrict__ mask, uint2* __restrict__ range) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const uint32_t key = pkey[p];
    if (p == 0 || pkey[p - 1] != key) range[key].x = (uint32_t)p;
    if (p == n_pairs - 1 || pkey[p + 1] != key) range[key].y = (uint32_t)(p + 1);
    const int view = view_of_tile(bp, (int)key);
    const uint32_t t = pkey[p] - (uint32_t)bp.tile_base[view];
    const uint32_t tiles_x = (uint32_t)bp.views[view].tiles_x;
    const uint64_t rc = __ldg(rect_sorted + pval[p]);
    const int x0 = (int)(t % (uint32_t)tiles_x) * DV_TILE, y0 = (int)(t / (uint32_t)tiles_x) * DV_TILE;
    const int u0 = (int)(rc & 0xffff) - x0, u1 = (int)((rc >> 16) & 0xffff) - x0;
    const int v0 = (int)((rc >> 32) & 0xffff) - y0, v1 = (int)(rc >> 48) - y0;
    uint32_t m = 0;
#pragma unroll
    for (int sy = 0; sy < 4; ++sy)
#pragma unroll
        for (int sx = 0; sx < 2; ++sx)
            if (u0 <= 8 * sx + 7 && u1 >= 8 * sx && v0 <= 4 * sy + 3 && v1 >= 4 * sy) m |= 1u << (sy * 2 + sx);
    mask[p] = (uint8_t)m;
}

// Heaviest tiles first: counting sort of tiles by floor(log2(list length + 1)),
// descending, so the longest CTAs start early and the short ones fill in behind
// them, within three groups that run as separate launches of the compositing
// kernel: the tiles that 5 or more actor clip boxes cover (buckets 64..95), those
// that 1 to 4 cover (32..63), the others (0..31).  The order inside a bucket does
// not matter (tiles are independent).
constexpr int TILE_BUCKETS = 96;

__device__ __forceinline__ int tile_bucket(const BatchParams& bp, const uint2* __restrict__ range, int t) {
    const uint2 r = range[t];
    const int b = 31 - __clz((int)(r.y - r.x) + 1);
    const int view = view_of_tile(bp, t);
    const int tl = t - bp.tile_base[view];
    const int tiles_x = bp.views[view].tiles_x;
    const int tx = tl % tiles_x, ty = tl / tiles_x;
    const OctParams* vo = bp.octs + view * bp.n_oct;
    int boxes = 0;
    for (int o = 1; o < bp.n_oct && boxes < 5; ++o) {
        const OctParams& P = vo[o];
        if (P.role == DV_ROLE_ACTOR && P.rect[0] <= tx && tx <= P.rect[2] && P.rect[1] <= ty && ty <= P.rect[3])
            ++boxes;
    }
    return b + (boxes >= 5 ? 64 : boxes > 0 ? 32 : 0);
}

__global__ void k_tile_count(const __grid_constant__ BatchParams bp, const uint2* __restrict__ range, int n_tiles,
                             uint32_t* __restrict__ cnt) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ uint32_t h[TILE_BUCKETS];
    if (threadIdx.x < TILE_BUCKETS) h[threadIdx.x] = 0;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) atomicAdd(&h[tile_bucket(bp, range, t)], 1u);
    __syncthreads();
    if (threadIdx.x < TILE_BUCKETS && h[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_tile_offsets(uint32_t* __restrict__ cnt_off) {
    pdl_wait();
    pdl_launch_dependents();
    // cnt_off[0..95] counts -> cnt_off[96..191] start of each bucket, from the heaviest bucket of the
    // first group down
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = TILE_BUCKETS - 1; b >= 0; --b) {
            cnt_off[TILE_BUCKETS + b] = run;
            run += cnt_off[b];
        }
    }
}

__global__ void k_tile_scatter(const __grid_constant__ BatchParams bp, const uint2* __restrict__ range, int n_tiles,
                               uint32_t* __restrict__ off, uint32_t* __restrict__ order) {
    pdl_wait();
    pdl_launch_dependents();
    // block-local ranks first, then one global reservation per (block, bucket)
    __shared__ uint32_t h[TILE_BUCKETS], base[TILE_BUCKETS];
    if (threadIdx.x < TILE_BUCKETS) h[threadIdx.x] = 0;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = t < n_tiles ? tile_bucket(bp, range, t) : -1;
    const uint32_t rank = b >= 0 ? atomicAdd(&h[b], 1u) : 0u;
    __syncthreads();
    if (threadIdx.x < TILE_BUCKETS && h[threadIdx.x])
        base[threadIdx.x] = atomicAdd(&off[threadIdx.x], h[threadIdx.x]);
    __syncthreads();
    if (b >= 0) order[base[b] + rank] = (uint32_t)t;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_tile_order(const BatchParams& bp, const uint2* tile_range, int n_tiles, uint32_t* scratch192,
                              uint32_t* order, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(scratch192, 0, 2 * TILE_BUCKETS * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    launch_pdl(k_tile_count, dim3(nblk(n_tiles, 256)), dim3(256), s, bp, tile_range, n_tiles, scratch192);
    count_launches(1);
    launch_pdl(k_tile_offsets, dim3(1), dim3(32), s, scratch192);
    count_launches(1);
    launch_pdl(k_tile_scatter, dim3(nblk(n_tiles, 256)), dim3(256), s, bp, tile_range, n_tiles,
               scratch192 + TILE_BUCKETS, order);
    count_launches(1);
    return cudaGetLastError();
}

// copies n counters into mapped host memory (system-scope stores, visible to the host once the
// stream has passed this kernel)
__global__ void k_publish(const uint64_t* __restrict__ src, volatile uint64_t* dst, int n, uint32_t* spin_err,
                          int flag_idx) {
    pdl_wait();
    pdl_launch_dependents();
    const int t = threadIdx.x;
    if (t < n) {
        uint64_t v = src[t];
        if (t == flag_idx && spin_err && atomicExch(spin_err, 0u)) v |= DV_FLAG_SPIN_TIMEOUT;
        dst[t] = v;
    }
    __threadfence_system();
}

cudaError_t launch_publish(const uint64_t* src, uint64_t* host_mapped_dst, int n, uint32_t* spin_err, int flag_idx,
                           cudaStream_t s) {
    launch_pdl(k_publish, dim3(1), dim3(32), s, src, host_mapped_dst, n, spin_err, flag_idx);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_project(const BatchParams& bp, uint32_t* cnt, uint64_t* rect, uint64_t* skey, uint32_t* vis,
                           uint32_t* flags, unsigned long long* totals, cudaStream_t s) {
    const int64_t n = bp.n_vox * bp.n_view;
    if (n <= 0) return cudaSuccess;
    launch_pdl(k_project, dim3(nblk(n, 256)), dim3(256), s, bp, cnt, rect, skey, vis, flags, totals);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint32_t* vis, const uint32_t* pos, const uint64_t* skey, int64_t n,
                           uint64_t* out_key, uint32_t* out_val, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    launch_pdl(k_compact, dim3(nblk(n, 256)), dim3(256), s, vis, pos, skey, n, out_key, out_val);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_records(const BatchParams& bp, const uint32_t* sorted_g, int64_t n_vis, const uint32_t* cnt,
                           const uint64_t* rect, VoxRec* rec, float4* nrm, uint32_t* cnt_sorted,
                           uint64_t* rect_sorted, cudaStream_t s) {
    if (n_vis <= 0) return cudaSuccess;
    launch_pdl(k_records, dim3(nblk(n_vis, 256)), dim3(256), s, bp, sorted_g, n_vis, cnt, rect, rec, nrm, cnt_sorted, rect_sorted);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_vis_start(const BatchParams& bp, const uint64_t* sorted_key, int64_t n_vis, uint32_t* vis_start,
                             cudaStream_t s) {
    if (n_vis <= 0) return cudaMemsetAsync(vis_start, 0, sizeof(uint32_t) * (bp.n_view * bp.n_oct + 1), s);
    launch_pdl(k_vis_start, dim3(nblk(n_vis, 256)), dim3(256), s, bp, sorted_key, n_vis, vis_start);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_emit(const BatchParams& bp, const uint64_t* off, const uint64_t* rect_sorted,
                        const uint32_t* sorted_g, int64_t n_vis, int64_t n_pairs, uint32_t* pair_key,
                        uint32_t* pair_val, cudaStream_t s) {
    if (n_vis <= 0 || n_pairs <= 0) return cudaSuccess;
    launch_pdl(k_emit, dim3(nblk(n_pairs, 256)), dim3(256), s, bp, off, rect_sorted, sorted_g, n_vis, n_pairs, pair_key, pair_val);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pair_mask_ranges(const BatchParams& bp, const uint32_t* pair_key, const uint32_t* pair_val,
                                    const uint64_t* rect_sorted, int64_t n_pairs, uint8_t* mask, uint2* tile_range,
                                    int n_tiles, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(tile_range, 0, sizeof(uint2) * (size_t)n_tiles, s);
    if (e != cudaSuccess || n_pairs <= 0) return e;
    launch_pdl(k_pair_mask, dim3(nblk(n_pairs, 256)), dim3(256), s, bp, pair_key, pair_val, rect_sorted, n_pairs, mask, tile_range);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dv
