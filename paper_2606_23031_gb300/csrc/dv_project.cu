// Per-voxel projection, render records and tile binning.
//
// All kernels run over every view of a render call at once (a view is one camera
// of one request, with its own actor poses); tiles are numbered globally.
//
// project  (one thread per (view, voxel) of every octree): leaf geometry from its key,
//          the 8 corners placed in the camera frame by the composed pose
//          (local -> world -> camera, Sec. 3.2), near/far culling, a conservative
//          screen rectangle of the box (clipped against the near plane) turned
//          into a tile rectangle, and the depth-order key.  The visible ones are
//          appended (one reservation per block) to the depth sort's input, whose
//          digit counts the same kernel takes; the last block to finish writes the
//          call's sizes into mapped host memory.
// records  (one thread per visible voxel, in depth-key order): 64-byte record
//          with the local box, the 8 raw densities and the view-dependent SH
//          colour for this camera; the block then writes the (tile, record) pairs
//          of its voxels, one per tile of each rectangle, at the offsets a
//          single-pass scan (look-back over earlier blocks) gives, counting the
//          pairs of every tile and the digits of the tile sort on the way.
// mask     which 8x4-pixel blocks of its tile each sorted pair touches, and the tile ranges.
// order    the tiles by list length (from the per-tile counts) within their actor-coverage group.
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
// Keys are unique (distinct leaves have distinct paths), so the order in which
// the projection appends them does not change the sorted result.
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

// Projection of (view, voxel) g: returns its tile count (0: not visible) and, when visible, its
// pixel rectangle and depth-order key.
__device__ __forceinline__ uint32_t project_voxel(const BatchParams& bp, int64_t g, uint64_t& rect,
                                                  uint64_t& skey, uint32_t* __restrict__ flags) {
    const int view = (int)(g / bp.n_vox);
    const int64_t gv = g - (int64_t)view * bp.n_vox;
    const int o = find_octree(bp, gv);
    const ViewParams& fp = bp.views[view];
    const OctParams& P = bp.octs[view * bp.n_oct + o];
    const int64_t v = gv - bp.vox_offset[o];
    const uint64_t key = P.key[v];
    const Leaf L = decode_leaf(P, key);
    if (L.level > P.max_level || L.i >> L.level || L.j >> L.level || L.k >> L.level) {
        atomicOr(flags, DV_FLAG_BAD_LEVEL);
        __threadfence();  // visible to the block that reports the flags
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
    // pixel rectangle (tiles are its pixels >> 4)
    rect = (uint64_t)pu0 | ((uint64_t)pu1 << 16) | ((uint64_t)pv0 << 32) | ((uint64_t)pv1 << 48);
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
    skey = ((uint64_t)view << bp.view_shift) | ((uint64_t)o << bp.oct_shift) | bsp;
    return n_tiles;
}

constexpr int MAX_KEY_PASSES = 8;  // 8-bit digits of a 64-bit key

// One thread per (view, voxel).  A block reserves one run of the sort input for its visible voxels
// (scal[0] counts them, scal[1] their pairs), adds the digits of their keys to key_hist
// [key_passes][256], and the block that finishes last copies scal[0..2] into host_out[0..2] (the
// device's wait-error word folded into the flags) and then `seq` into host_out[3], so the host learns
// the sizes from this kernel alone, as soon as they are final.  scal[3] counts finished blocks.
// Block 0 also clears the call's five work words.
__global__ void __launch_bounds__(256) k_project(const __grid_constant__ BatchParams bp, uint32_t* __restrict__ cnt,
                                                 uint64_t* __restrict__ rect, uint64_t* __restrict__ out_key,
                                                 uint32_t* __restrict__ out_g, uint32_t* __restrict__ key_hist,
                                                 int key_passes, unsigned long long* __restrict__ scal,
                                                 volatile uint64_t* host_out, uint64_t seq,
                                                 uint32_t* __restrict__ spin_err, unsigned long long* __restrict__ work) {
    pdl_wait();
    pdl_launch_dependents();
    if (blockIdx.x == 0 && threadIdx.x < 5) work[threadIdx.x] = 0ull;
    __shared__ uint32_t h[MAX_KEY_PASSES][256];
    __shared__ uint32_t s_wv[8];
    __shared__ unsigned long long s_wp[8];
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_nv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + tid;  // view * n_vox + voxel
    uint64_t rc = 0, key = 0;
    uint32_t c = 0;
    if (g < bp.n_vox * bp.n_view) c = project_voxel(bp, g, rc, key, reinterpret_cast<uint32_t*>(scal + 2));
    const unsigned bal = __ballot_sync(0xffffffffu, c != 0);
    unsigned long long np = c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) np += __shfl_down_sync(0xffffffffu, np, off);
    if (lane == 0) {
        s_wv[warp] = __popc(bal);
        s_wp[warp] = np;
    }
    for (int i = tid; i < key_passes * 256; i += 256) (&h[0][0])[i] = 0u;
    __syncthreads();
    if (tid == 0) {
        uint32_t nv = 0;
        unsigned long long pp = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t x = s_wv[w];
            s_wv[w] = nv;  // exclusive offsets of the warps
            nv += x;
            pp += s_wp[w];
        }
        s_nv = nv;
        s_base = nv ? atomicAdd(scal + 0, (unsigned long long)nv) : 0ull;
        if (pp) atomicAdd(scal + 1, pp);
    }
    __syncthreads();
    if (s_nv) {
        if (c) {
            const unsigned long long q = s_base + s_wv[warp] + __popc(bal & ((1u << lane) - 1u));
            out_key[q] = key;
            out_g[q] = (uint32_t)g;
            cnt[g] = c;
            rect[g] = rc;
            for (int p = 0; p < key_passes; ++p) atomicAdd(&h[p][(uint32_t)(key >> (8 * p)) & 255u], 1u);
        }
        __syncthreads();
        for (int i = tid; i < key_passes * 256; i += 256) {
            const uint32_t x = (&h[0][0])[i];
            if (x) atomicAdd(key_hist + i, x);
        }
    }
    // the last block to finish sees every block's counts (each block's totals come from its thread 0,
    // a flag from the thread that set it, after its own fence)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned long long done = atomicAdd(scal + 3, 1ull);
        if (done == gridDim.x - 1) {
            __threadfence();
            const uint64_t nv = atomicAdd(scal + 0, 0ull), pp = atomicAdd(scal + 1, 0ull);
            uint64_t fl = atomicOr(reinterpret_cast<unsigned long long*>(scal + 2), 0ull);
            if (spin_err && atomicExch(spin_err, 0u)) fl |= DV_FLAG_SPIN_TIMEOUT;
            host_out[0] = nv;
            host_out[1] = pp;
            host_out[2] = fl;
            __threadfence_system();
            host_out[3] = seq;
            __threadfence_system();
        }
    }
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

// (view, octree) group of a depth key: view * n_oct + octree
__device__ __forceinline__ int key_group(const BatchParams& bp, uint64_t k) {
    const int view = (int)(k >> bp.view_shift);
    const int o = (int)((k >> bp.oct_shift) & ((1ull << (bp.view_shift - bp.oct_shift)) - 1));
    return view * bp.n_oct + o;
}

constexpr int MAX_PAIR_PASSES = 4;  // 8-bit digits of a 32-bit tile index
constexpr unsigned long long LB_INC = 1ull << 63, LB_AGG = 1ull << 62, LB_VAL = LB_AGG - 1ull;

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}

// One thread per visible voxel in depth-key order, blocks taken in order from a counter.
//  1. the voxel's render record (and normal), its rectangle in depth order, and the start of its
//     (view, octree) group in vis_start;
//  2. the block's pair offsets: a block scan of the tile counts, then the block's first pair from
//     a look-back over the earlier blocks' published counts (the block reads 256 predecessors at a
//     time; an inclusive one ends the walk; every spin is bounded);
//  3. the block's pairs, spread over all its threads (a pair finds its voxel by binary search in
//     the block's offsets), with the tile-sort digits and the per-tile pair counts.
__global__ void __launch_bounds__(256) k_records_emit(
    const __grid_constant__ BatchParams bp, const uint32_t* __restrict__ sorted_g,
    const uint64_t* __restrict__ sorted_key, int64_t n_vis, int64_t n_pairs, const uint32_t* __restrict__ cnt,
    const uint64_t* __restrict__ rect, VoxRec* __restrict__ rec, float4* __restrict__ nrm,
    uint64_t* __restrict__ rect_sorted, uint32_t* __restrict__ vis_start, uint32_t* __restrict__ pkey,
    uint32_t* __restrict__ pval, uint32_t* __restrict__ pair_hist, int pair_passes, uint32_t* __restrict__ tile_cnt,
    unsigned long long* __restrict__ lb_status, uint32_t* __restrict__ ticket, uint32_t* __restrict__ call_err,
    uint32_t* __restrict__ dev_err, int spin_limit) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ uint32_t s_blk;
    __shared__ uint32_t s_off[256];
    __shared__ uint64_t s_rc[256];
    __shared__ int32_t s_tb[256], s_tx[256];
    __shared__ uint32_t s_ws[8];
    __shared__ uint32_t s_inc[8];
    __shared__ unsigned long long s_part[8];
    __shared__ unsigned long long s_excl;
    __shared__ uint32_t h[MAX_PAIR_PASSES][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_blk = atomicAdd(ticket, 1u);
    for (int i = tid; i < pair_passes * 256; i += 256) (&h[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t blk = s_blk;
    const int64_t r = (int64_t)blk * 256 + tid;
    uint32_t c = 0;
    if (r < n_vis) {
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
        // rho = c0 + c1 x + c2 y + c3 z + c4 xy + c5 xz + c6 yz + c7 xyz, from corner c = x + 2y + 4z,
        // stored as (c0, c3, c1, c5), (c2, c6, c4, c7) for the compositing kernels' packed FMAs
        const float p1 = da.y - da.x, p2 = da.z - da.x, p3 = db.x - da.x;
        const float p4 = (da.w - da.z) - p1, p5 = (db.y - db.x) - p1, p6 = (db.z - db.x) - p2;
        const float p7 = ((db.w - db.z) - (db.y - db.x)) - ((da.w - da.z) - p1);
        R.v[1] = make_float4(da.x, p3, p1, p5);
        R.v[2] = make_float4(p2, p6, p4, p7);
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
        c = cnt[g];
        const uint64_t rc = rect[g];
        rect_sorted[r] = rc;
        s_rc[tid] = rc;
        s_tb[tid] = bp.tile_base[view];
        s_tx[tid] = bp.views[view].tiles_x;
        // start of every (view, octree) group in depth order
        const int grp = key_group(bp, sorted_key[r]);
        const int prev = r > 0 ? key_group(bp, sorted_key[r - 1]) : -1;
        for (int q = prev + 1; q <= grp; ++q) vis_start[q] = (uint32_t)r;
        if (r == n_vis - 1)
            for (int q = grp + 1; q <= bp.n_view * bp.n_oct; ++q) vis_start[q] = (uint32_t)n_vis;
    }
    // block exclusive scan of the tile counts
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_ws[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t x = s_ws[w];
        wbase += w < warp ? x : 0u;
        total += x;
    }
    s_off[tid] = wbase + incl - c;
    // the block's first pair: publish the block's count, then look back over the earlier blocks,
    // 256 at a time (thread j reads block blk - 1 - j); the nearest inclusive count ends the walk
    unsigned long long* mine = lb_status + blk;
    if (tid == 0) *(volatile unsigned long long*)mine = (blk == 0 ? LB_INC : LB_AGG) | total;
    unsigned long long excl = 0;
    if (blk > 0) {
        for (int64_t t = (int64_t)blk - 1; t >= 0; t -= 256) {
            const int64_t i = t - tid;
            unsigned long long v = i >= 0 ? lb_load(lb_status + i) : LB_INC;
            int spins = 0;
            while (!(v & (LB_INC | LB_AGG)) && ++spins < spin_limit) v = lb_load(lb_status + i);
            const bool lost = !(v & (LB_INC | LB_AGG));
            const unsigned inc = __ballot_sync(0xffffffffu, (v & LB_INC) != 0);
            if (lane == 0) s_inc[warp] = inc ? warp * 32 + __ffs(inc) - 1 : 256;
            if (__syncthreads_or(lost)) {
                if (tid == 0) {
                    atomicOr(call_err, 1u);
                    atomicOr(dev_err, 1u);
                }
                break;
            }
            int stop = 256;  // nearest inclusive predecessor in this window
#pragma unroll
            for (int w = 0; w < 8; ++w) stop = min(stop, (int)s_inc[w]);
            unsigned long long x = tid <= stop ? (v & LB_VAL) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) s_part[warp] = x;
            __syncthreads();
#pragma unroll
            for (int w = 0; w < 8; ++w) excl += s_part[w];
            __syncthreads();  // s_inc and s_part are rewritten by the next window
            if (stop < 256) break;
        }
        if (tid == 0) *(volatile unsigned long long*)mine = LB_INC | (excl + total);
    }
    if (tid == 0) s_excl = excl;
    __syncthreads();
    const unsigned long long first = s_excl;
    const int64_t left = n_vis - (int64_t)blk * 256;
    const int nb = left < 256 ? (int)left : 256;
    for (uint32_t i = tid; i < total; i += 256) {
        int lo = 0, hi = nb - 1;  // last voxel of the block whose first pair is <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= i)
                lo = mid;
            else
                hi = mid - 1;
        }
        const uint64_t rc = s_rc[lo];
        const uint32_t tx0 = (rc & 0xffff) >> 4, tx1 = ((rc >> 16) & 0xffff) >> 4, ty0 = ((rc >> 32) & 0xffff) >> 4;
        const uint32_t w = tx1 - tx0 + 1;
        const uint32_t k = i - s_off[lo];
        const uint32_t tile = (uint32_t)s_tb[lo] + (ty0 + k / w) * (uint32_t)s_tx[lo] + tx0 + k % w;
        const unsigned long long p = first + i;
        if (p < (unsigned long long)n_pairs) {  // only a timed-out look-back can leave the range
            pkey[p] = tile;
            pval[p] = blk * 256u + (uint32_t)lo;
        }
        atomicAdd(tile_cnt + tile, 1u);
        for (int q = 0; q < pair_passes; ++q) atomicAdd(&h[q][(tile >> (8 * q)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = tid; i < pair_passes * 256; i += 256) {
        const uint32_t x = (&h[0][0])[i];
        if (x) atomicAdd(pair_hist + i, x);
    }
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
// touches (bit sy * 2 + sx), and the [first, end) range of every tile that has pairs, from the key
// boundaries.  Thread 0 also copies the call's sort flag into its mapped host status word (the sorts
// have all completed when this kernel runs).
__global__ void k_pair_mask(const __grid_constant__ BatchParams bp, const uint32_t* __restrict__ pkey,
                            const uint32_t* __restrict__ pval, const uint64_t* __restrict__ rect_sorted,
                            int64_t n_pairs, int64_t n_vis, uint8_t* __restrict__ mask, uint2* __restrict__ range,
                            const uint64_t* __restrict__ sort_err, volatile uint64_t* status_out) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && status_out) {
        *status_out = *(const volatile uint64_t*)sort_err;
        __threadfence_system();
    }
    if (p >= n_pairs) return;
    const uint32_t key = pkey[p];
    if (key < (uint32_t)bp.n_tiles) {  // always, unless a sort wait timed out
        if (p == 0 || pkey[p - 1] != key) range[key].x = (uint32_t)p;
        if (p == n_pairs - 1 || pkey[p + 1] != key) range[key].y = (uint32_t)(p + 1);
    }
    const int view = view_of_tile(bp, (int)key);
    const uint32_t t = key - (uint32_t)bp.tile_base[view];
    const uint32_t tiles_x = (uint32_t)bp.views[view].tiles_x;
    const uint32_t v = min(pval[p], (uint32_t)(n_vis - 1));  // in range unless a sort wait timed out
    const uint64_t rc = __ldg(rect_sorted + v);
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

__device__ __forceinline__ int tile_bucket(const BatchParams& bp, uint32_t n_pairs, int t) {
    const int b = 31 - __clz((int)n_pairs + 1);
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

// one thread per tile: its bucket (kept in bucket[t]) into the global bucket counts hist[96]; a tile
// without pairs gets the empty range (the pair-mask kernel wrote the others)
__global__ void __launch_bounds__(256) k_tile_count(const __grid_constant__ BatchParams bp,
                                                    const uint32_t* __restrict__ tile_cnt, int n_tiles,
                                                    uint8_t* __restrict__ bucket, uint2* __restrict__ range,
                                                    uint32_t* __restrict__ hist) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ uint32_t h[TILE_BUCKETS];
    if (threadIdx.x < TILE_BUCKETS) h[threadIdx.x] = 0;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) {
        const uint32_t c = tile_cnt[t];
        if (c == 0) range[t] = make_uint2(0u, 0u);
        const int b = tile_bucket(bp, c, t);
        bucket[t] = (uint8_t)b;
        atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < TILE_BUCKETS && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// one thread per tile: each block turns the 96 bucket counts into bucket starts, heaviest bucket of
// the first group first, then reserves one run per (block, bucket) from the cursors
__global__ void __launch_bounds__(256) k_tile_scatter(const uint8_t* __restrict__ bucket, int n_tiles,
                                                      const uint32_t* __restrict__ hist,
                                                      uint32_t* __restrict__ cursor, uint32_t* __restrict__ order) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ uint32_t start[TILE_BUCKETS], h[TILE_BUCKETS], base[TILE_BUCKETS];
    const int tid = threadIdx.x;
    if (tid < TILE_BUCKETS) h[tid] = 0;
    if (tid == 0) {
        uint32_t run = 0;
        for (int b = TILE_BUCKETS - 1; b >= 0; --b) {
            start[b] = run;
            run += hist[b];
        }
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + tid;
    const int b = t < n_tiles ? bucket[t] : -1;
    const uint32_t rank = b >= 0 ? atomicAdd(&h[b], 1u) : 0u;
    __syncthreads();
    if (tid < TILE_BUCKETS && h[tid]) base[tid] = start[tid] + atomicAdd(&cursor[tid], h[tid]);
    __syncthreads();
    if (b >= 0) order[base[b] + rank] = (uint32_t)t;
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

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

int key_passes(int n_bits) { return (n_bits + 7) / 8; }

cudaError_t launch_publish(const uint64_t* src, uint64_t* host_mapped_dst, int n, uint32_t* spin_err, int flag_idx,
                           cudaStream_t s) {
    launch_pdl(k_publish, dim3(1), dim3(32), s, src, host_mapped_dst, n, spin_err, flag_idx);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_project(const BatchParams& bp, uint32_t* cnt, uint64_t* rect, uint64_t* out_key, uint32_t* out_g,
                           uint32_t* key_hist, int key_bits, unsigned long long* scal, uint64_t* host_out, uint64_t seq,
                           uint32_t* spin_err, unsigned long long* work, cudaStream_t s) {
    const int64_t n = bp.n_vox * bp.n_view;
    const int passes = key_passes(key_bits);
    if (passes > MAX_KEY_PASSES) return cudaErrorInvalidValue;
    // with no voxel at all, one empty block still clears the work words and reports the (zero) sizes
    launch_pdl(k_project, dim3(n > 0 ? nblk(n, 256) : 1u), dim3(256), s, bp, cnt, rect, out_key, out_g, key_hist,
               passes, scal, (volatile uint64_t*)host_out, seq, spin_err, work);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_records_emit(const BatchParams& bp, const uint32_t* sorted_g, const uint64_t* sorted_key,
                                int64_t n_vis, int64_t n_pairs, const uint32_t* cnt, const uint64_t* rect,
                                VoxRec* rec, float4* nrm, uint64_t* rect_sorted, uint32_t* vis_start,
                                uint32_t* pair_key, uint32_t* pair_val, uint32_t* pair_hist, int tile_bits,
                                uint32_t* tile_cnt, unsigned long long* lb_status, uint32_t* ticket,
                                uint32_t* call_err, uint32_t* dev_err, cudaStream_t s) {
    if (n_vis <= 0) return cudaMemsetAsync(vis_start, 0, sizeof(uint32_t) * (bp.n_view * bp.n_oct + 1), s);
    const int passes = key_passes(tile_bits);
    if (passes > MAX_PAIR_PASSES || !call_err || !dev_err) return cudaErrorInvalidValue;
    launch_pdl(k_records_emit, dim3(nblk(n_vis, 256)), dim3(256), s, bp, sorted_g, sorted_key, n_vis, n_pairs, cnt,
               rect, rec, nrm, rect_sorted, vis_start, pair_key, pair_val, pair_hist, passes, tile_cnt, lb_status,
               ticket, call_err, dev_err, (int)(1 << 22));
    count_launches(1);
    return cudaGetLastError();
}

int64_t records_emit_blocks(int64_t n_vis) { return (n_vis + 255) / 256; }

cudaError_t launch_pair_mask(const BatchParams& bp, const uint32_t* pair_key, const uint32_t* pair_val,
                             const uint64_t* rect_sorted, int64_t n_pairs, int64_t n_vis, uint8_t* mask,
                             uint2* tile_range, const uint64_t* sort_err, uint64_t* status_host, cudaStream_t s) {
    if (n_pairs <= 0) return launch_publish(sort_err, status_host, 1, nullptr, -1, s);
    launch_pdl(k_pair_mask, dim3(nblk(n_pairs, 256)), dim3(256), s, bp, pair_key, pair_val, rect_sorted, n_pairs,
               n_vis, mask, tile_range, sort_err, (volatile uint64_t*)status_host);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const BatchParams& bp, const uint32_t* tile_cnt, int n_tiles, uint2* range,
                              uint8_t* bucket, uint32_t* scratch192, uint32_t* order, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    launch_pdl(k_tile_count, dim3(nblk(n_tiles, 256)), dim3(256), s, bp, tile_cnt, n_tiles, bucket, range,
               scratch192);
    count_launches(1);
    launch_pdl(k_tile_scatter, dim3(nblk(n_tiles, 256)), dim3(256), s, (const uint8_t*)bucket, n_tiles,
               (const uint32_t*)scratch192, scratch192 + TILE_BUCKETS, order);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dv
