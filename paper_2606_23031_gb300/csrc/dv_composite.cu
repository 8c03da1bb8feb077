// Front-to-back compositing over each ray's voxel segments (forward) and its
// replay with gradients (backward), plus the SH-colour backward.
//
// One CTA renders one 16x16 tile, one thread per pixel (Sec. 3.4, Alg. 1):
//  * The tile's pair list is grouped by octree and, inside an octree, sorted
//    front to back for every ray of the camera (depth-order key, see
//    dv_project.cu).  The background sub-list is streamed through shared
//    memory in batches of 256 records that every pixel of the tile tests.
//  * Each pixel splits its ray into background and actor intervals with the
//    actor clip boxes (slab test in each actor's frame, reached through the
//    inverse pose; the box entered first owns any overlap).  Intervals are
//    found lazily: the next one is the unvisited box with the smallest entry
//    distance among those still ahead.
//  * While walking the background list, a hit that reaches past the next
//    actor's entry first composites its part in front of the box, then the
//    pixel walks that actor's sub-list (clipped to the actor's interval),
//    then continues with the remainder of the background voxel behind the
//    box.  The running state (C, D, T) is carried across every border, so the
//    composite equals the global front-to-back order of all segments.
//  * Per segment: trilinear interpolation of the raw corner densities at K
//    midpoints, exponential-linear activation, tau = l/K sum sigma,
//    alpha = 1 - exp(-tau), C += T alpha c, D += T alpha (t0+t1)/2,
//    T *= 1 - alpha, stop once T < eps_stop.
//  * The backward replays exactly the forward's segment sequence (same code,
//    stopping after the forward's segment count) front to back.  With
//    w_k = T_k alpha_k it uses dC/dtau_k = T_{k+1} c_k - sum_{j>k} w_j c_j where the
//    suffix sum is C_final - (prefix through k), so no division by (1 - alpha)
//    and no reverse traversal is needed.  Gradients of the background records
//    are reduced across the warp (all lanes visit the same record together)
//    before one atomic per value; actor-walk gradients use per-lane atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dv_internal.cuh"

namespace dv {

namespace {

constexpr int BATCH = DV_BLOCK;
constexpr int GSTRIDE = 12;  // per-record gradient slots: 8 densities, 3 colour, 1 pad

struct Pix {
    float C0, C1, C2, D, T;
    uint32_t n;
    uint32_t tests, boxes;  // work counters: voxel slab tests, actor box tests
    bool done;
};

struct Bwd {
    // upstream gradient, forward results, running prefix sums
    float g0, g1, g2, gD, gA;
    float Cf0, Cf1, Cf2, Df, Tend;
    float P0, P1, P2, PD;
    uint32_t nmax;
};

struct ActInt {
    int o;
    float a, b;
};

__device__ __forceinline__ float act_fn(float x, int act) {
    if (act == DV_ACT_IDENTITY) return x;
    return x > 1.1f ? x : 1.1f * expf(fmaf(x, 0.90909090909090909f, -1.0f));
}

__device__ __forceinline__ float act_grad(float x, int act) {
    if (act == DV_ACT_IDENTITY) return 1.0f;
    return x > 1.1f ? 1.0f : expf(fmaf(x, 0.90909090909090909f, -1.0f));
}

__device__ __forceinline__ void rotate(const float* A, const float* x, float* y) {
#pragma unroll
    for (int r = 0; r < 3; ++r) y[r] = fmaf(A[r * 3 + 0], x[0], fmaf(A[r * 3 + 1], x[1], A[r * 3 + 2] * x[2]));
}

__device__ __forceinline__ bool slab_cube(const float* o, const float* inv, float4 g, float& t0, float& t1) {
    const float lo[3] = {g.x, g.y, g.z};
    float a = -INFINITY, b = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ta = (lo[k] - o[k]) * inv[k];
        const float tb = (lo[k] + g.w - o[k]) * inv[k];
        a = fmaxf(a, fminf(ta, tb));
        b = fminf(b, fmaxf(ta, tb));
    }
    t0 = a;
    t1 = b;
    return a < b;
}

__device__ __forceinline__ bool slab_box(const float* o, const float* inv, const float* h, float& t0, float& t1) {
    float a = -INFINITY, b = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ta = (-h[k] - o[k]) * inv[k];
        const float tb = (h[k] - o[k]) * inv[k];
        a = fmaxf(a, fminf(ta, tb));
        b = fminf(b, fmaxf(ta, tb));
    }
    t0 = a;
    t1 = b;
    return a < b;
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// optical depth of the segment [t0, t1] through one voxel; optionally d tau / d dens[c]
template <bool GRAD>
__device__ __forceinline__ float seg_tau(float4 g, float4 da, float4 db, const float* o, const float* d, float t0,
                                         float t1, int K, int act, float* dtd) {
    const float h = (t1 - t0) / (float)K;
    const float is = 1.0f / g.w;
    float tau = 0.0f;
    if (GRAD) {
#pragma unroll
        for (int c = 0; c < 8; ++c) dtd[c] = 0.0f;
    }
    for (int k = 0; k < K; ++k) {
        const float t = fmaf((float)k + 0.5f, h, t0);
        const float x = __saturatef((fmaf(t, d[0], o[0]) - g.x) * is);
        const float y = __saturatef((fmaf(t, d[1], o[1]) - g.y) * is);
        const float z = __saturatef((fmaf(t, d[2], o[2]) - g.z) * is);
        const float e00 = lerpf(da.x, da.y, x), e10 = lerpf(da.z, da.w, x);
        const float e01 = lerpf(db.x, db.y, x), e11 = lerpf(db.z, db.w, x);
        const float rho = lerpf(lerpf(e00, e10, y), lerpf(e01, e11, y), z);
        tau += act_fn(rho, act);
        if (GRAD) {
            const float s = act_grad(rho, act) * h;
            const float x0 = 1.0f - x, y0 = 1.0f - y, z0 = 1.0f - z;
            dtd[0] = fmaf(s, x0 * y0 * z0, dtd[0]);
            dtd[1] = fmaf(s, x * y0 * z0, dtd[1]);
            dtd[2] = fmaf(s, x0 * y * z0, dtd[2]);
            dtd[3] = fmaf(s, x * y * z0, dtd[3]);
            dtd[4] = fmaf(s, x0 * y0 * z, dtd[4]);
            dtd[5] = fmaf(s, x * y0 * z, dtd[5]);
            dtd[6] = fmaf(s, x0 * y * z, dtd[6]);
            dtd[7] = fmaf(s, x * y * z, dtd[7]);
        }
    }
    return tau * h;
}

// Composites one segment; in the backward also adds this segment's gradient
// into acc[0..10] (8 densities, 3 colour channels).
template <bool BWD>
__device__ __forceinline__ void add_segment(Pix& ps, Bwd& bw, const FrameParams& fp, float4 g, float4 da, float4 db,
                                            float4 col, const float* o, const float* d, float t0, float t1,
                                            float* acc) {
    float dtd[8];
    const float tau = seg_tau<BWD>(g, da, db, o, d, t0, t1, fp.K, fp.activation, dtd);
    const float alpha = -expm1f(-tau);
    const float w = ps.T * alpha;
    const float mid = 0.5f * (t0 + t1);
    ps.C0 = fmaf(w, col.x, ps.C0);
    ps.C1 = fmaf(w, col.y, ps.C1);
    ps.C2 = fmaf(w, col.z, ps.C2);
    ps.D = fmaf(w, mid, ps.D);
    ps.T = ps.T * (1.0f - alpha);
    ps.n += 1;
    if (BWD) {
        const float Tn = ps.T;
        float gt = bw.gA * bw.Tend;
        gt = fmaf(bw.g0, fmaf(Tn, col.x, -(bw.Cf0 - ps.C0)), gt);
        gt = fmaf(bw.g1, fmaf(Tn, col.y, -(bw.Cf1 - ps.C1)), gt);
        gt = fmaf(bw.g2, fmaf(Tn, col.z, -(bw.Cf2 - ps.C2)), gt);
        gt = fmaf(bw.gD, fmaf(Tn, mid, -(bw.Df - ps.D)), gt);
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = fmaf(gt, dtd[c], acc[c]);
        acc[8] = fmaf(bw.g0, w, acc[8]);
        acc[9] = fmaf(bw.g1, w, acc[9]);
        acc[10] = fmaf(bw.g2, w, acc[10]);
        if (ps.n >= bw.nmax) ps.done = true;
    } else {
        if (ps.T < fp.eps_stop) ps.done = true;
    }
}

// next actor interval ahead of tau_cur (first-entered box owns overlaps)
__device__ __forceinline__ ActInt next_interval(const FrameParams& fp, const int16_t* tact, int n_ta, const float* dc,
                                                float tau_cur) {
    ActInt r;
    r.o = -1;
    r.a = INFINITY;
    r.b = 0.0f;
    for (int q = 0; q < n_ta; ++q) {
        const OctParams& P = fp.oc[tact[q]];
        float d[3], inv[3], a, b;
        rotate(P.A, dc, d);
        inv[0] = 1.0f / d[0];
        inv[1] = 1.0f / d[1];
        inv[2] = 1.0f / d[2];
        if (!slab_box(P.o_loc, inv, P.clip_half, a, b)) continue;
        a = fmaxf(a, fp.near_);
        b = fminf(b, fp.far_);
        if (!(b > a) || !(b > tau_cur)) continue;
        if (a < r.a) {
            r.o = tact[q];
            r.a = a;
            r.b = b;
        }
    }
    if (r.o >= 0) r.a = fmaxf(r.a, tau_cur);
    return r;
}

template <bool BWD>
__device__ __forceinline__ void atomic_grad(float* grad_rec, uint32_t r, const float* acc) {
    float* gp = grad_rec + (size_t)r * GSTRIDE;
#pragma unroll
    for (int c = 0; c < 11; ++c)
        if (acc[c] != 0.0f) atomicAdd(gp + c, acc[c]);
}

// walk one actor's sub-list of the tile, clipped to its interval
template <bool BWD>
__device__ __noinline__ void walk_actor(Pix& ps, Bwd& bw, const FrameParams& fp, const ActInt& it,
                                        const uint32_t* __restrict__ pval, const VoxRec* __restrict__ rec,
                                        uint32_t q0, uint32_t q1, const float* dc, float* grad_rec) {
    const OctParams& P = fp.oc[it.o];
    float d[3], inv[3];
    rotate(P.A, dc, d);
    inv[0] = 1.0f / d[0];
    inv[1] = 1.0f / d[1];
    inv[2] = 1.0f / d[2];
    const float o[3] = {P.o_loc[0], P.o_loc[1], P.o_loc[2]};
    for (uint32_t q = q0; q < q1 && !ps.done; ++q) {
        ps.tests += 1;
        const uint32_t r = __ldg(pval + q);
        const float4* R = rec[r].v;
        const float4 g = __ldg(R);
        float t0, t1;
        if (!slab_cube(o, inv, g, t0, t1)) continue;
        t0 = fmaxf(t0, it.a);
        t1 = fminf(t1, it.b);
        if (!(t1 > t0)) continue;
        float acc[11];
#pragma unroll
        for (int c = 0; c < 11; ++c) acc[c] = 0.0f;
        add_segment<BWD>(ps, bw, fp, g, __ldg(R + 1), __ldg(R + 2), __ldg(R + 3), o, d, t0, t1, acc);
        if (BWD) atomic_grad<BWD>(grad_rec, r, acc);
    }
}

template <bool BWD>
__global__ void __launch_bounds__(DV_BLOCK) k_composite(const __grid_constant__ FrameParams fp,
                                                        const VoxRec* __restrict__ rec,
                                                        const uint32_t* __restrict__ pval,
                                                        const uint2* __restrict__ tile_range,
                                                        const uint32_t* __restrict__ vis_start,
                                                        float* __restrict__ out_rgb, float* __restrict__ out_depth,
                                                        float* __restrict__ out_alpha, uint32_t* __restrict__ n_seg,
                                                        float* __restrict__ t_final, const float* __restrict__ g_rgb,
                                                        const float* __restrict__ g_depth,
                                                        const float* __restrict__ g_alpha,
                                                        float* __restrict__ grad_rec,
                                                        unsigned long long* __restrict__ work) {
    __shared__ float4 s_rec[BATCH][4];
    __shared__ uint32_t s_r[BATCH];
    __shared__ uint32_t s_sub[DV_MAX_OCTREES + 1];
    __shared__ int16_t s_act[DV_MAX_OCTREES];
    __shared__ int s_nact;

    const int tile = blockIdx.x;
    const int tx = tile % fp.tiles_x, ty = tile / fp.tiles_x;
    const uint2 rg = tile_range[tile];
    const int tid = threadIdx.x;
    if (tid <= fp.n_oct) {
        const uint32_t key = vis_start[tid];
        uint32_t lo = rg.x, hi = rg.y;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(pval + mid) < key)
                lo = mid + 1;
            else
                hi = mid;
        }
        s_sub[tid] = lo;
    }
    if (tid == 0) {
        int n = 0;
        for (int o = 1; o < fp.n_oct; ++o) {
            const OctParams& P = fp.oc[o];
            if (P.role == DV_ROLE_ACTOR && P.rect[0] <= tx && tx <= P.rect[2] && P.rect[1] <= ty && ty <= P.rect[3])
                s_act[n++] = (int16_t)o;
        }
        s_nact = n;
    }
    __syncthreads();

    const int u = tx * DV_TILE + (tid & (DV_TILE - 1));
    const int v = ty * DV_TILE + (tid >> 4);
    const bool valid = u < fp.W && v < fp.H;
    const int64_t pix = (int64_t)v * fp.W + u;

    float dc[3];
    {
        const float x = ((float)u + 0.5f - fp.cx) / fp.fx;
        const float y = ((float)v + 0.5f - fp.cy) / fp.fy;
        const float in = rsqrtf(fmaf(x, x, fmaf(y, y, 1.0f)));
        dc[0] = x * in;
        dc[1] = y * in;
        dc[2] = in;
    }
    const OctParams& B = fp.oc[0];
    float db_[3], ib[3];
    rotate(B.A, dc, db_);
    ib[0] = 1.0f / db_[0];
    ib[1] = 1.0f / db_[1];
    ib[2] = 1.0f / db_[2];
    const float ob[3] = {B.o_loc[0], B.o_loc[1], B.o_loc[2]};

    Pix ps;
    ps.C0 = ps.C1 = ps.C2 = ps.D = 0.0f;
    ps.T = 1.0f;
    ps.n = 0;
    ps.tests = 0;
    ps.boxes = 0;
    ps.done = !valid;
    Bwd bw;
    if (BWD) {
        if (valid) {
            bw.g0 = g_rgb ? g_rgb[pix * 3 + 0] : 0.0f;
            bw.g1 = g_rgb ? g_rgb[pix * 3 + 1] : 0.0f;
            bw.g2 = g_rgb ? g_rgb[pix * 3 + 2] : 0.0f;
            bw.gD = g_depth ? g_depth[pix] : 0.0f;
            bw.gA = g_alpha ? g_alpha[pix] : 0.0f;
            bw.Cf0 = out_rgb[pix * 3 + 0];
            bw.Cf1 = out_rgb[pix * 3 + 1];
            bw.Cf2 = out_rgb[pix * 3 + 2];
            bw.Df = out_depth[pix];
            bw.Tend = t_final[pix];
            bw.nmax = n_seg[pix];
            if (bw.nmax == 0) ps.done = true;
        } else {
            bw.nmax = 0;
        }
    }
    const int n_ta = s_nact;
    float tau_cur = fp.near_;
    ActInt nxt;
    nxt.o = -1;
    if (valid && n_ta > 0) {
        nxt = next_interval(fp, s_act, n_ta, dc, tau_cur);
        ps.boxes += n_ta;
    }

    const uint32_t bg0 = s_sub[0], bg1 = s_sub[1];
    for (uint32_t base = bg0; base < bg1; base += BATCH) {
        const uint32_t cnt = min((uint32_t)BATCH, bg1 - base);
        if ((uint32_t)tid < cnt) {
            const uint32_t r = __ldg(pval + base + tid);
            const float4* R = rec[r].v;
            s_rec[tid][0] = __ldg(R);
            s_rec[tid][1] = __ldg(R + 1);
            s_rec[tid][2] = __ldg(R + 2);
            s_rec[tid][3] = __ldg(R + 3);
            s_r[tid] = r;
        }
        __syncthreads();
        for (uint32_t j = 0; j < cnt; ++j) {
            if (!BWD && ps.done) break;
            float acc[11];
            if (BWD) {
#pragma unroll
                for (int c = 0; c < 11; ++c) acc[c] = 0.0f;
            }
            bool contributed = false;
            const float4 g = s_rec[j][0];
            float t_in, t_out;
            if (!ps.done) ps.tests += 1;
            if (!ps.done && slab_cube(ob, ib, g, t_in, t_out)) {
                t_in = fmaxf(t_in, fp.near_);
                t_out = fminf(t_out, fp.far_);
                if (t_out > t_in) {
                    const float4 da = s_rec[j][1], dd = s_rec[j][2], col = s_rec[j][3];
                    float cur = fmaxf(t_in, tau_cur);
                    while (nxt.o >= 0 && nxt.a < t_out && !ps.done) {
                        if (nxt.a > cur) {
                            add_segment<BWD>(ps, bw, fp, g, da, dd, col, ob, db_, cur, nxt.a, acc);
                            contributed = true;
                            if (ps.done) break;
                        }
                        walk_actor<BWD>(ps, bw, fp, nxt, pval, rec, s_sub[nxt.o], s_sub[nxt.o + 1], dc, grad_rec);
                        tau_cur = nxt.b;
                        cur = fmaxf(cur, nxt.b);
                        nxt = next_interval(fp, s_act, n_ta, dc, tau_cur);
                        ps.boxes += n_ta;
                    }
                    if (!ps.done && t_out > cur) {
                        add_segment<BWD>(ps, bw, fp, g, da, dd, col, ob, db_, cur, t_out, acc);
                        contributed = true;
                    }
                }
            }
            if (BWD) {
                // all lanes visit record j together: reduce across the warp, one atomic per value
                const unsigned any = __ballot_sync(0xffffffffu, contributed);
                if (any) {
#pragma unroll
                    for (int c = 0; c < 11; ++c) {
                        float x = acc[c];
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
                        acc[c] = x;
                    }
                    if ((tid & 31) == 0) atomic_grad<BWD>(grad_rec, s_r[j], acc);
                }
            }
        }
        if (__syncthreads_count(!ps.done) == 0) break;
    }
    // actor intervals behind the last background hit
    while (nxt.o >= 0 && !ps.done) {
        walk_actor<BWD>(ps, bw, fp, nxt, pval, rec, s_sub[nxt.o], s_sub[nxt.o + 1], dc, grad_rec);
        tau_cur = nxt.b;
        nxt = next_interval(fp, s_act, n_ta, dc, tau_cur);
        ps.boxes += n_ta;
    }
    if (!BWD && work) {
        unsigned long long t = ps.tests, b = ps.boxes, n = ps.n;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            t += __shfl_down_sync(0xffffffffu, t, off);
            b += __shfl_down_sync(0xffffffffu, b, off);
            n += __shfl_down_sync(0xffffffffu, n, off);
        }
        if ((tid & 31) == 0) {
            atomicAdd(work + 0, t);
            atomicAdd(work + 1, b);
            atomicAdd(work + 2, n);
        }
    }
    if (!BWD && valid) {
        out_rgb[pix * 3 + 0] = ps.C0;
        out_rgb[pix * 3 + 1] = ps.C1;
        out_rgb[pix * 3 + 2] = ps.C2;
        out_depth[pix] = ps.D;
        out_alpha[pix] = 1.0f - ps.T;
        n_seg[pix] = ps.n;
        t_final[pix] = ps.T;
    }
}

// ---------------------------------------------------------------------------
// SH colour backward + scatter of the per-record gradients to the caller's arrays
// ---------------------------------------------------------------------------

__device__ __forceinline__ void sh_basis_f(int deg, float x, float y, float z, float* b) {
    // same basis as the records kernel (real SH, degree <= 3)
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

struct ShBwdOct {
    float o_loc[3];
    int32_t sh_degree;
    int64_t vox_offset;
    const float* sh;
    float* d_dens;
    float* d_sh;
};

struct ShBwdParams {
    int32_t n_oct;
    ShBwdOct oc[DV_MAX_OCTREES];
};

__global__ void __launch_bounds__(256) k_sh_bwd(const __grid_constant__ ShBwdParams sp,
                                                const uint32_t* __restrict__ sorted_g, int64_t n_vis,
                                                const VoxRec* __restrict__ rec, const float* __restrict__ grad_rec) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_vis) return;
    const uint32_t gidx = sorted_g[r];
    int lo = 0, hi = sp.n_oct - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sp.oc[mid].vox_offset <= (int64_t)gidx)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ShBwdOct& P = sp.oc[lo];
    const int64_t v = (int64_t)gidx - P.vox_offset;
    const float* gr = grad_rec + (size_t)r * GSTRIDE;
    if (P.d_dens) {
        float* dd = P.d_dens + v * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) dd[c] += gr[c];
    }
    const float gc0 = gr[8], gc1 = gr[9], gc2 = gr[10];
    if (!P.d_sh || (gc0 == 0.0f && gc1 == 0.0f && gc2 == 0.0f)) return;
    const float4 g = rec[r].v[0];
    float gx = g.x + 0.5f * g.w - P.o_loc[0];
    float gy = g.y + 0.5f * g.w - P.o_loc[1];
    float gz = g.z + 0.5f * g.w - P.o_loc[2];
    const float gl = sqrtf(gx * gx + gy * gy + gz * gz);
    const float ig = gl > 0.0f ? 1.0f / gl : 0.0f;
    gx *= ig;
    gy *= ig;
    gz *= ig;
    float b[16];
    sh_basis_f(P.sh_degree, gx, gy, gz, b);
    const int nsh = (P.sh_degree + 1) * (P.sh_degree + 1);
    const float* shv = P.sh + v * nsh * 3;
    float c0 = 0.5f, c1 = 0.5f, c2 = 0.5f;
    for (int q = 0; q < nsh; ++q) {
        c0 = fmaf(b[q], shv[q * 3 + 0], c0);
        c1 = fmaf(b[q], shv[q * 3 + 1], c1);
        c2 = fmaf(b[q], shv[q * 3 + 2], c2);
    }
    const float m0 = c0 > 0.0f ? gc0 : 0.0f, m1 = c1 > 0.0f ? gc1 : 0.0f, m2 = c2 > 0.0f ? gc2 : 0.0f;
    float* ds = P.d_sh + v * nsh * 3;
    for (int q = 0; q < nsh; ++q) {
        ds[q * 3 + 0] += b[q] * m0;
        ds[q * 3 + 1] += b[q] * m1;
        ds[q * 3 + 2] += b[q] * m2;
    }
}

}  // namespace

cudaError_t launch_composite_fwd(const FrameParams& fp, const VoxRec* rec, const uint32_t* pair_val,
                                 const uint2* tile_range, const uint32_t* vis_start, float* rgb, float* depth,
                                 float* alpha, uint32_t* n_seg, float* t_final, unsigned long long* work,
                                 cudaStream_t s) {
    const int n_tiles = fp.tiles_x * fp.tiles_y;
    if (n_tiles <= 0) return cudaSuccess;
    k_composite<false><<<n_tiles, DV_BLOCK, 0, s>>>(fp, rec, pair_val, tile_range, vis_start, rgb, depth, alpha,
                                                    n_seg, t_final, nullptr, nullptr, nullptr, nullptr, work);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_composite_bwd(const FrameParams& fp, const VoxRec* rec, const uint32_t* pair_val,
                                 const uint2* tile_range, const uint32_t* vis_start, const float* rgb,
                                 const float* depth, const uint32_t* n_seg, const float* t_final, const float* g_rgb,
                                 const float* g_depth, const float* g_alpha, float* grad_rec, cudaStream_t s) {
    const int n_tiles = fp.tiles_x * fp.tiles_y;
    if (n_tiles <= 0) return cudaSuccess;
    k_composite<true><<<n_tiles, DV_BLOCK, 0, s>>>(fp, rec, pair_val, tile_range, vis_start, const_cast<float*>(rgb),
                                                   const_cast<float*>(depth), nullptr, const_cast<uint32_t*>(n_seg),
                                                   const_cast<float*>(t_final), g_rgb, g_depth, g_alpha, grad_rec,
                                                   nullptr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sh_bwd(const FrameParams& fp, const uint32_t* sorted_g, int64_t n_vis, const VoxRec* rec,
                          const float* grad_rec, float* const* d_dens, float* const* d_sh, cudaStream_t s) {
    if (n_vis <= 0) return cudaSuccess;
    ShBwdParams sp;
    sp.n_oct = fp.n_oct;
    for (int o = 0; o < fp.n_oct; ++o) {
        const OctParams& P = fp.oc[o];
        ShBwdOct& q = sp.oc[o];
        q.o_loc[0] = P.o_loc[0];
        q.o_loc[1] = P.o_loc[1];
        q.o_loc[2] = P.o_loc[2];
        q.sh_degree = P.sh_degree;
        q.vox_offset = P.vox_offset;
        q.sh = P.sh;
        q.d_dens = d_dens ? d_dens[o] : nullptr;
        q.d_sh = d_sh ? d_sh[o] : nullptr;
    }
    k_sh_bwd<<<(unsigned)((n_vis + 255) / 256), 256, 0, s>>>(sp, sorted_g, n_vis, rec, grad_rec);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dv
