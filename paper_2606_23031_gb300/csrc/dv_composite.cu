// Front-to-back compositing over each ray's voxel segments (forward) and its
// replay with gradients (backward), plus the SH-colour backward.
//
// Each CTA renders half of a 16x16 tile (16x8 pixels, 4 warps of 8x4 pixels),
// one thread per pixel, tiles taken heaviest first (Sec. 3.4, Alg. 1):
//  * The tile's pair list is grouped by octree and, inside an octree, sorted
//    front to back for every ray of the camera (depth-order key, see
//    dv_project.cu).
//  * Each pixel splits its ray into background and actor intervals with the
//    actor clip boxes (slab test in each actor's frame, reached through the
//    inverse pose; the box entered first owns any overlap).
//  * Every sub-list (each actor's, the background's) streams through a two-slot
//    shared-memory ring (cp.async, one batch ahead); each warp visits, in list
//    order and in lockstep, the records that touch its 8x4 pixel block.
//  * Phase 1: for every actor of the tile, every lane composites the segments
//    inside its own interval of that actor into a partial (C_A, D_A, T_A)
//    starting from T = 1.
//  * Phase 2: the background sub-list.  A background hit that reaches past the
//    next actor's entry composites its part in front of the box, then applies
//    that actor's partial with the running transmittance (C += T C_A,
//    D += T D_A, T *= T_A), then continues behind the box.  If T T_A < eps_stop
//    the ray must stop inside the actor: the lane records its state and stops.
//  * Phase 3: lanes that stop inside an actor replay that actor's sub-list in
//    lockstep from the recorded state with the exact stop rule.
//    Since T only decreases along the ray, applying a whole partial is exact
//    unless the stop falls inside it, which is exactly when T T_A < eps_stop.
//  * Per segment: trilinear interpolation of the raw corner densities at K
//    midpoints, exponential-linear activation, tau = l/K sum sigma,
//    alpha = 1 - exp(-tau), C += T alpha c, D += T alpha (t0+t1)/2,
//    T *= 1 - alpha, stop once T < eps_stop.
//  * The backward runs the same three phases (identical arithmetic, so the same
//    stops).  With w_k = T_k alpha_k it uses
//    dC/dtau_k = T_{k+1} c_k - sum_{j>k} w_j c_j, the suffix sum being
//    C_final - (prefix through k), so it needs no division by (1 - alpha) and
//    no reverse traversal.  Phase 2 records, for every actor interval reached,
//    the prefix state at its entry; phase 3 then replays every reached actor
//    interval with gradients from that state.  Gradients of records visited in
//    lockstep are reduced across the warp before the atomics.
//  * Tiles with more actors than lockstep slots (4, or 16 where 5 or more boxes
//    cover the tile) handle the extra actors with a per-lane walk of the actor's
//    sub-list (correct, but divergent).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dv_internal.cuh"

namespace dv {

namespace {

constexpr int CT_THREADS = 128;  // half a tile per CTA
// per-record gradient slots: 8 densities, 3 colour (+ 3 normal with normals), padded to 16 bytes
template <bool NRM>
struct GradLayout {
    static constexpr int NV = NRM ? 14 : 11;      // values per record
    static constexpr int STRIDE = NRM ? 16 : 12;  // floats per record row
};
// lockstep actor slots of the two actor variants: tiles that 1 to 4 actor boxes cover, and tiles
// that 5 or more cover (beyond 8, the remaining actors take the per-thread walk)
constexpr int NTA_SMALL = 4;
constexpr int NTA_LARGE = 8;

struct PixBase {
    float C0, C1, C2, D, T;
    float R;  // residual form of the backward: sum over the composited segments of w (dL/dC . c + dL/dD mid)
    uint32_t n;
    uint32_t tests, boxes;  // work counters: voxel slab tests, actor box tests
    bool done;
};
template <bool NRM>
struct Pix : PixBase {};
template <>
struct Pix<true> : PixBase {
    float N0, N1, N2;  // normal state
};

struct BwdBase {
    // upstream gradient and the forward's results
    float g0, g1, g2, gD, gA;
    float Cf0, Cf1, Cf2, Df, Tend;
    float base;  // dL/dA T_end - (dL/dC . C_final + dL/dD D_final [+ dL/dN . N_final]), for the residual form
};
template <bool NRM>
struct Bwd : BwdBase {};
template <>
struct Bwd<true> : BwdBase {
    float gN0, gN1, gN2, Nf0, Nf1, Nf2;  // normal state: upstream gradient and final value
};

// per-lane writer of the composited segments' (voxel, weight) list (weights export)
struct ExportSink {
    uint32_t* vid;             // [total] voxel index within the view's concatenated octrees
    float* w;                  // [total] T alpha
    const uint32_t* sorted_g;  // record -> view * n_vox + voxel
    int64_t base, voff;        // first slot of this pixel; view * n_vox
    uint32_t n, lim;           // written so far; this pixel's slots
};

struct ActInt {
    int o;  // octree index (-1: none)
    int q;  // slot in the tile's actor list
    float a, b;
};

// 2^x on the SFU (ex2.approx.ftz: relative error about 2^-22)
__device__ __forceinline__ float ex2_sfu(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// exponential-linear activation: x above 1.1, 1.1 exp(x/1.1 - 1) below (C1 at 1.1).  The exponential
// branch is one SFU power of two, 1.1 exp(x/1.1 - 1) = 2^(x / (1.1 ln 2) + (ln 1.1 - 1) / ln 2), and
// its slope exp(x/1.1 - 1) is the same power divided by 1.1.
__device__ __forceinline__ float explin_low(float x) {
    return ex2_sfu(fmaf(x, 1.3115409462626941f, -1.3051915171390283f));
}

__device__ __forceinline__ float act_fn(float x, int act) {
    if (act == DV_ACT_IDENTITY) return x;
    return x > 1.1f ? x : explin_low(x);
}

__device__ __forceinline__ float act_grad(float x, int act) {
    if (act == DV_ACT_IDENTITY) return 1.0f;
    return x > 1.1f ? 1.0f : explin_low(x) * 0.90909090909090909f;
}

__device__ __forceinline__ void rotate(const float* A, const float* x, float* y) {
#pragma unroll
    for (int r = 0; r < 3; ++r) y[r] = fmaf(A[r * 3 + 0], x[0], fmaf(A[r * 3 + 1], x[1], A[r * 3 + 2] * x[2]));
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Inverse ray direction, also split by sign, so that the slab test takes each axis's
// entry and exit plane without a min/max.  |d| is kept at or above 1e-20, so every
// product stays finite: a ray parallel to a slab gets entry and exit times of order
// 1e20 of the right signs instead of infinities (and NaN where inf - inf would meet).
struct InvDir {
    float inv[3];  // 1 / d
    float ip[3];   // 1 / d where d > 0, else 0
    float in[3];   // 1 / d where d < 0, else 0
};

__device__ __forceinline__ InvDir inv_dir(const float* d) {
    InvDir r;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float dk = fabsf(d[k]) < 1e-20f ? copysignf(1e-20f, d[k]) : d[k];
        r.inv[k] = 1.0f / dk;
        r.ip[k] = dk > 0.0f ? r.inv[k] : 0.0f;
        r.in[k] = dk < 0.0f ? r.inv[k] : 0.0f;
    }
    return r;
}

// Ray / voxel slab test.  g = (min corner - ray origin, size): along axis k the ray
// crosses the min plane at g_k / d_k and the max plane at (g_k + size) / d_k; which of
// the two it enters by follows from the sign of d_k.  The x and y axes go through packed two-lane
// multiplies and FMAs (the same roundings as scalar ones, half the instructions).
__device__ __forceinline__ bool slab_cube(const InvDir& v, float4 g, float& t0, float& t1) {
    const float2 ww = make_float2(g.w, g.w);
    const float2 ta = __fmul2_rn(make_float2(g.x, g.y), make_float2(v.inv[0], v.inv[1]));
    const float2 en = __ffma2_rn(ww, make_float2(v.in[0], v.in[1]), ta);
    const float2 ex = __ffma2_rn(ww, make_float2(v.ip[0], v.ip[1]), ta);
    const float tz = g.z * v.inv[2];
    t0 = max3f(en.x, en.y, fmaf(g.w, v.in[2], tz));
    t1 = min3f(ex.x, ex.y, fmaf(g.w, v.ip[2], tz));
    return t0 < t1;
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


// optical depth of the segment [t0, t1] through one voxel (da, db: the record's density polynomial);
// optionally d tau / d dens[c] for the raw corner densities
// KS > 0: K known at compile time (KS); KS == 0: K from the launch.  With GRAD and a single sample
// (KS == 1), d tau / d dens[c] = s w_c(x, y, z) is left factored: sxyz receives (s, x, y, z), the
// activation's slope times the step and the sample's voxel coordinates, and dtd is not written.
template <bool GRAD, int KS>
__device__ __forceinline__ float seg_tau(float4 da, float4 db, float is, const float* rel, const float* d, float t0,
                                         float t1, int K_rt, float inv_k_rt, int act, float* dtd, float* sxyz) {
    const int K = KS > 0 ? KS : K_rt;
    const float inv_k = KS == 1 ? 1.0f : inv_k_rt;
    const float h = (t1 - t0) * inv_k;
    float tau = 0.0f;
    if (GRAD && KS != 1) {
#pragma unroll
        for (int c = 0; c < 8; ++c) dtd[c] = 0.0f;
    }
    for (int k = 0; k < K; ++k) {
        const float t = fmaf((float)k + 0.5f, h, t0);
        // voxel-local coordinates of the sample o + t d: (t d - (min - o)) / size
        const float x = __saturatef(fmaf(t, d[0], -rel[0]) * is);
        const float y = __saturatef(fmaf(t, d[1], -rel[1]) * is);
        const float z = __saturatef(fmaf(t, d[2], -rel[2]) * is);
        // the record holds the trilinear field as a polynomial (da = (c0, c3, c1, c5), db = (c2, c6, c4,
        // c7)): rho = (c0 + c1 x) + y (c2 + c4 x) + z ((c3 + c5 x) + y (c6 + c7 x)), the two x-linear
        // pairs and the two y steps taken as packed two-lane FMAs (same roundings as the scalar form)
        const float2 xx = make_float2(x, x);
        const float2 pA = __ffma2_rn(make_float2(da.z, da.w), xx, make_float2(da.x, da.y));
        const float2 pB = __ffma2_rn(make_float2(db.z, db.w), xx, make_float2(db.x, db.y));
        const float2 qq = __ffma2_rn(pB, make_float2(y, y), pA);
        const float rho = fmaf(qq.y, z, qq.x);
        tau += act_fn(rho, act);
        if (GRAD && KS == 1) {
            sxyz[0] = act_grad(rho, act) * h;
            sxyz[1] = x;
            sxyz[2] = y;
            sxyz[3] = z;
        } else if (GRAD) {
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

// Front-to-back compositing of one segment of optical depth tau; returns its weight T alpha.
template <bool NRM>
__device__ __forceinline__ float composite_step(Pix<NRM>& ps, float tau, float4 col, float4 nv, float t0, float t1) {
    const float e = __expf(-tau);  // transmittance of the segment
    const float alpha = 1.0f - e;
    const float w = ps.T * alpha;
    const float mid = 0.5f * (t0 + t1);
    ps.C0 = fmaf(w, col.x, ps.C0);
    ps.C1 = fmaf(w, col.y, ps.C1);
    ps.C2 = fmaf(w, col.z, ps.C2);
    ps.D = fmaf(w, mid, ps.D);
    if constexpr (NRM) {
        ps.N0 = fmaf(w, nv.x, ps.N0);
        ps.N1 = fmaf(w, nv.y, ps.N1);
        ps.N2 = fmaf(w, nv.z, ps.N2);
    }
    ps.T = ps.T * e;
    ps.n += 1;
    return w;
}

template <bool NRM>
__device__ __forceinline__ void composite_tau(Pix<NRM>& ps, float tau, float4 col, float4 nv, float t0, float t1,
                                              float eps_stop) {
    composite_step<NRM>(ps, tau, col, nv, t0, t1);
    if (ps.T < eps_stop) ps.done = true;
}

// d L / d dens[c] of one segment, added into acc[0..7], from gt = d L / d tau
template <int KS>
__device__ __forceinline__ void seg_density_grad(float gt, const float* dtd, const float* sxyz, float* acc) {
    if constexpr (KS == 1) {
        // gt s w_c(x, y, z): the trilinear weights with gt s folded into the y-z products; corners c and
        // c + 1 (x = 0 and 1) are accumulated as one packed two-lane FMA
        const float a = gt * sxyz[0];
        const float x = sxyz[1], y = sxyz[2], z = sxyz[3];
        const float2 xw = make_float2(1.0f - x, x);
        const float2 ay = __fmul2_rn(make_float2(a, a), make_float2(1.0f - y, y));
        const float2 cz0 = __fmul2_rn(ay, make_float2(1.0f - z, 1.0f - z));
        const float2 cz1 = __fmul2_rn(ay, make_float2(z, z));
        float2 r;
        r = __ffma2_rn(xw, make_float2(cz0.x, cz0.x), make_float2(acc[0], acc[1])); acc[0] = r.x; acc[1] = r.y;
        r = __ffma2_rn(xw, make_float2(cz0.y, cz0.y), make_float2(acc[2], acc[3])); acc[2] = r.x; acc[3] = r.y;
        r = __ffma2_rn(xw, make_float2(cz1.x, cz1.x), make_float2(acc[4], acc[5])); acc[4] = r.x; acc[5] = r.y;
        r = __ffma2_rn(xw, make_float2(cz1.y, cz1.y), make_float2(acc[6], acc[7])); acc[6] = r.x; acc[7] = r.y;
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = fmaf(gt, dtd[c], acc[c]);
    }
}

// Composites one segment (with the stop test when STOP); with GRAD also adds
// this segment's gradient into acc[0..10] (8 densities, 3 colour channels).
// RF (backward only): the residual form.  The gradient of tau_k only needs the upstream-weighted
// sums, dL/dtau_k = T_{k+1} s_k - (K - R_k) + dL/dA T_end with s_k = dL/dC . c_k + dL/dD mid_k
// (+ dL/dN . n_k), K the same sum over the final images and R_k = sum_{j <= k} w_j s_j; so the lane
// carries the one scalar R instead of the prefix colour, depth (and normal).
template <bool GRAD, bool STOP, int KS, bool NRM, bool WEX = false, bool RF = false>
__device__ __forceinline__ void add_segment(Pix<NRM>& ps, const Bwd<NRM>& bw, const BatchParams& bp, float4 da, float4 db,
                                            float4 col, float4 nv, const float* rel, const float* d, float t0,
                                            float t1, float* acc, uint32_t r = 0, ExportSink* ex = nullptr) {
    float dtd[8], sxyz[4];
    const float tau = seg_tau<GRAD, KS>(da, db, col.w, rel, d, t0, t1, bp.K, bp.inv_k, bp.activation, dtd, sxyz);
    if constexpr (RF) {
        // (without GRAD: an actor's partial in the backward, R only)
        const float e = __expf(-tau);
        const float w = ps.T * (1.0f - e);
        const float mid = 0.5f * (t0 + t1);
        float s = fmaf(bw.g0, col.x, fmaf(bw.g1, col.y, fmaf(bw.g2, col.z, bw.gD * mid)));
        if constexpr (NRM) s = fmaf(bw.gN0, nv.x, fmaf(bw.gN1, nv.y, fmaf(bw.gN2, nv.z, s)));
        ps.R = fmaf(w, s, ps.R);
        ps.T = ps.T * e;
        ps.n += 1;
        if constexpr (GRAD) {
            const float gt = fmaf(ps.T, s, bw.base + ps.R);
            seg_density_grad<KS>(gt, dtd, sxyz, acc);
            acc[8] = fmaf(bw.g0, w, acc[8]);
            acc[9] = fmaf(bw.g1, w, acc[9]);
            acc[10] = fmaf(bw.g2, w, acc[10]);
            if constexpr (NRM) {
                acc[11] = fmaf(bw.gN0, w, acc[11]);
                acc[12] = fmaf(bw.gN1, w, acc[12]);
                acc[13] = fmaf(bw.gN2, w, acc[13]);
            }
        }
        if (STOP && ps.T < bp.eps_stop) ps.done = true;
        return;
    }
    const float w = composite_step<NRM>(ps, tau, col, nv, t0, t1);
    if constexpr (WEX) {
        if (ex->n < ex->lim) {
            ex->vid[ex->base + ex->n] = (uint32_t)((int64_t)ex->sorted_g[r] - ex->voff);
            ex->w[ex->base + ex->n] = w;
        }
        ex->n += 1;
    }
    if (GRAD) {
        const float mid = 0.5f * (t0 + t1);
        const float Tn = ps.T;
        float gt = bw.gA * bw.Tend;
        gt = fmaf(bw.g0, fmaf(Tn, col.x, -(bw.Cf0 - ps.C0)), gt);
        gt = fmaf(bw.g1, fmaf(Tn, col.y, -(bw.Cf1 - ps.C1)), gt);
        gt = fmaf(bw.g2, fmaf(Tn, col.z, -(bw.Cf2 - ps.C2)), gt);
        gt = fmaf(bw.gD, fmaf(Tn, mid, -(bw.Df - ps.D)), gt);
        if constexpr (NRM) {
            gt = fmaf(bw.gN0, fmaf(Tn, nv.x, -(bw.Nf0 - ps.N0)), gt);
            gt = fmaf(bw.gN1, fmaf(Tn, nv.y, -(bw.Nf1 - ps.N1)), gt);
            gt = fmaf(bw.gN2, fmaf(Tn, nv.z, -(bw.Nf2 - ps.N2)), gt);
            acc[11] = fmaf(bw.gN0, w, acc[11]);
            acc[12] = fmaf(bw.gN1, w, acc[12]);
            acc[13] = fmaf(bw.gN2, w, acc[13]);
        }
        seg_density_grad<KS>(gt, dtd, sxyz, acc);
        acc[8] = fmaf(bw.g0, w, acc[8]);
        acc[9] = fmaf(bw.g1, w, acc[9]);
        acc[10] = fmaf(bw.g2, w, acc[10]);
    }
    if (STOP && ps.T < bp.eps_stop) ps.done = true;
}

// One backward step in residual form with one sample, for a lane that meets the record at most once
// (a plain tile, or one actor interval): [u0, u1] is the lane's segment, the empty segment [0, 0] for a
// lane that misses or has finished (zero optical depth, weight and gradient, state unchanged).  The
// record's gradient values (8 densities, 3 colour, + 3 normal) are written into acc, not added, so the
// caller clears nothing and the warp runs it without branches once any lane hits.
template <bool NRM>
__device__ __forceinline__ void bwd_single_step(Pix<NRM>& ps, const Bwd<NRM>& bw, const BatchParams& bp, float4 g,
                                                float4 da, float4 dd, float4 col, float4 nv, const float* d, float u0,
                                                float u1, bool hit, float* acc) {
    const float rel[3] = {g.x, g.y, g.z};
    float sxyz[4];
    const float tau = seg_tau<true, 1>(da, dd, col.w, rel, d, u0, u1, bp.K, bp.inv_k, bp.activation, nullptr, sxyz);
    const float e = __expf(-tau);
    const float w = ps.T * (1.0f - e);
    const float mid = 0.5f * (u0 + u1);
    float sg = fmaf(bw.g0, col.x, fmaf(bw.g1, col.y, fmaf(bw.g2, col.z, bw.gD * mid)));
    if constexpr (NRM) sg = fmaf(bw.gN0, nv.x, fmaf(bw.gN1, nv.y, fmaf(bw.gN2, nv.z, sg)));
    ps.R = fmaf(w, sg, ps.R);
    ps.T = ps.T * e;
    ps.n += hit ? 1u : 0u;
    const float gt = fmaf(ps.T, sg, bw.base + ps.R);
    const float a = gt * sxyz[0];
    const float x = sxyz[1], y = sxyz[2], z = sxyz[3];
    const float2 xw = make_float2(1.0f - x, x);
    const float2 ay = __fmul2_rn(make_float2(a, a), make_float2(1.0f - y, y));
    const float2 cz0 = __fmul2_rn(ay, make_float2(1.0f - z, 1.0f - z));
    const float2 cz1 = __fmul2_rn(ay, make_float2(z, z));
    float2 r;
    r = __fmul2_rn(xw, make_float2(cz0.x, cz0.x));
    acc[0] = r.x;
    acc[1] = r.y;
    r = __fmul2_rn(xw, make_float2(cz0.y, cz0.y));
    acc[2] = r.x;
    acc[3] = r.y;
    r = __fmul2_rn(xw, make_float2(cz1.x, cz1.x));
    acc[4] = r.x;
    acc[5] = r.y;
    r = __fmul2_rn(xw, make_float2(cz1.y, cz1.y));
    acc[6] = r.x;
    acc[7] = r.y;
    acc[8] = bw.g0 * w;
    acc[9] = bw.g1 * w;
    acc[10] = bw.g2 * w;
    if constexpr (NRM) {
        acc[NRM ? 11 : 0] = bw.gN0 * w;
        acc[NRM ? 12 : 0] = bw.gN1 * w;
        acc[NRM ? 13 : 0] = bw.gN2 * w;
    }
    if (ps.T < bp.eps_stop) ps.done = true;
}

// next actor interval ahead of tau_cur (first-entered box owns overlaps)
__device__ __forceinline__ ActInt next_interval(const OctParams* __restrict__ vo, float t_near, float t_far,
                                                const int16_t* tact, int n_ta, const float* dc, float tau_cur) {
    ActInt r;
    r.o = -1;
    r.q = -1;
    r.a = INFINITY;
    r.b = 0.0f;
    for (int q = 0; q < n_ta; ++q) {
        const OctParams& P = vo[tact[q]];
        float d[3], inv[3], a, b;
        rotate(P.A, dc, d);
        inv[0] = 1.0f / d[0];
        inv[1] = 1.0f / d[1];
        inv[2] = 1.0f / d[2];
        if (!slab_box(P.o_loc, inv, P.clip_half, a, b)) continue;
        a = fmaxf(a, t_near);
        b = fminf(b, t_far);
        if (!(b > a) || !(b > tau_cur)) continue;
        if (a < r.a) {
            r.o = tact[q];
            r.q = q;
            r.a = a;
            r.b = b;
        }
    }
    if (r.o >= 0) r.a = fmaxf(r.a, tau_cur);
    return r;
}

template <bool NRM>
__device__ __forceinline__ void atomic_grad(float* grad_rec, uint32_t r, const float* acc) {
    float* gp = grad_rec + (size_t)r * GradLayout<NRM>::STRIDE;
#pragma unroll
    for (int c = 0; c < GradLayout<NRM>::NV; ++c)
        if (acc[c] != 0.0f) atomicAdd(gp + c, acc[c]);
}

// Sum of acc[0..NV-1] over the warp, transposed.  Each butterfly level (lane distance 16, 8, 4, 2,
// 1) splits the values the lane still holds into a first half (kept by the lanes without that
// distance's bit) and the rest (kept by the others), exchanging the half it gives up: NV = 11 takes
// 6 + 3 + 2 + 1 + 1 = 13 shuffles (14 values: 15).  Afterwards every value's total sits in exactly
// one lane, which adds it to the record's gradient slot.
template <int N, int D>
__device__ __forceinline__ void fold_level(float* v, int lane, int& idx, int& nreal) {
    if constexpr (D >= 1) {
        constexpr int H = (N + 1) / 2;
        const bool up = lane & D;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const float lo = v[i];
            const float hi = (H + i < N) ? v[H + i] : 0.0f;
            v[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, D);
        }
        idx += up ? H : 0;
        nreal = up ? max(nreal - H, 0) : min(nreal, H);
        fold_level<H, D / 2>(v, lane, idx, nreal);
    }
}

template <int NV>
__device__ __forceinline__ void warp_reduce_add(const float* acc, float* gp) {
    const int lane = threadIdx.x & 31;
    float v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = acc[c];
    int idx = 0, nreal = NV;
    fold_level<NV, 16>(v, lane, idx, nreal);
    if (nreal > 0 && v[0] != 0.0f) atomicAdd(gp + idx, v[0]);
}

// Record of pair q.  Every pair's record is below n_vis unless a sort's bounded wait ran out (the
// call is then reported as timed out); the clamp keeps the reads and gradient atomics in range.
__device__ __forceinline__ uint32_t rec_index(const BatchParams& bp, const uint32_t* __restrict__ pval, uint32_t q) {
    return min(__ldg(pval + q), (uint32_t)(bp.n_vis - 1));
}

// Per-lane walk of one actor's sub-list (divergent; only for actors beyond the
// NTA lockstep slots).
template <bool GRAD, int KS, bool NRM, bool WEX>
__device__ __noinline__ void walk_actor_lane(Pix<NRM>& ps, const Bwd<NRM>& bw, const BatchParams& bp,
                                             const OctParams* __restrict__ vo, const ActInt& it,
                                             const uint32_t* __restrict__ pval, const uint8_t* __restrict__ pmask,
                                             uint32_t wbit, const VoxRec* __restrict__ rec, uint32_t q0, uint32_t q1,
                                             const float* dc, float* grad_rec, ExportSink* ex) {
    const OctParams& P = vo[it.o];
    float d[3];
    rotate(P.A, dc, d);
    const InvDir inv = inv_dir(d);
    for (uint32_t q = q0; q < q1 && !ps.done; ++q) {
        if (!(__ldg(pmask + q) & wbit)) continue;
        ps.tests += 1;
        const uint32_t r = rec_index(bp, pval, q);
        const float4* R = rec[r].v;
        const float4 g = __ldg(R);
        float t0, t1;
        const float rel[3] = {g.x, g.y, g.z};
        if (!slab_cube(inv, g, t0, t1)) continue;
        t0 = fmaxf(t0, it.a);
        t1 = fminf(t1, it.b);
        if (!(t1 > t0)) continue;
        float acc[GradLayout<NRM>::NV];
#pragma unroll
        for (int c = 0; c < GradLayout<NRM>::NV; ++c) acc[c] = 0.0f;
        const float4 nv = NRM ? __ldg(bp.nrm + r) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        add_segment<GRAD, true, KS, NRM, WEX, GRAD>(ps, bw, bp, __ldg(R + 1), __ldg(R + 2), __ldg(R + 3), nv, rel, d, t0,
                                              t1, acc, r, ex);
        if (GRAD) atomic_grad<NRM>(grad_rec, r, acc);
    }
}

// 16-byte asynchronous global -> shared copy (L2 only), and its group fences
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// per-lane actor bookkeeping in shared memory, slot q < NTA:
//   s_iv[q][0/1][lane]  = the lane's owned interval [a, b) of that actor (a > b: none)
//   s_st[q][0..4][lane] = phase 1: partial (C0, C1, C2, D, T); phase 2 overwrites it with the
//                         state at the interval's entry (C0, C1, C2, D, T) when it is replayed
//   s_st[q][5][lane]    = phase 1: partial segment count; phase 2: 0 not reached,
//                         1 partial applied, 2 stop inside (replay)
//   s_st[q][6..8][lane] = with normals: the partial normal state N_A, then N at the entry

#ifndef DV_FWD_MIN_BLOCKS
#define DV_FWD_MIN_BLOCKS 5  // resident CTAs per SM the forward is compiled for
#endif
#ifndef DV_BWD_MIN_BLOCKS
#define DV_BWD_MIN_BLOCKS 4
#endif
#ifndef DV_PLAIN_MIN_BLOCKS
#define DV_PLAIN_MIN_BLOCKS 8  // the variant for tiles without actors (64 registers)
#endif

// BWD: replay with gradients.  WEX: replay that writes every composited segment's (voxel,
// weight) into the pixel's slots of the weights export (no outputs, no gradients).
// NTA: lockstep actor slots (0: the tile is covered by no actor clip box).  Tiles that no box covers
// (most of a frame) run the variant without the actor machinery: no interval walk, partials or
// replays, no per-pixel actor state in shared memory, and about half the registers, so about twice
// the resident warps per SM.  Tiles that many boxes cover get 16 slots, the others 4.
template <bool BWD, int KS, bool NRM, bool WEX, int NTA>
__global__ void __launch_bounds__(CT_THREADS, NTA ? ((BWD || WEX) ? DV_BWD_MIN_BLOCKS : DV_FWD_MIN_BLOCKS)
                                                  : DV_PLAIN_MIN_BLOCKS) k_composite(const __grid_constant__ BatchParams bp,
                                                        const VoxRec* __restrict__ rec,
                                                        const uint32_t* __restrict__ pval,
                                                        const uint8_t* __restrict__ pmask,
                                                        const uint2* __restrict__ tile_range,
                                                        const uint32_t* __restrict__ vis_start,
                                                        const uint32_t* __restrict__ tile_order,
                                                        uint32_t* __restrict__ n_seg,
                                                        float* __restrict__ t_final, const float* __restrict__ g_rgb,
                                                        const float* __restrict__ g_depth,
                                                        const float* __restrict__ g_alpha,
                                                        const float* __restrict__ g_normal,
                                                        float* __restrict__ grad_rec,
                                                        unsigned long long* __restrict__ work,
                                                        const int64_t* __restrict__ ex_off,
                                                        uint32_t* __restrict__ ex_vid, float* __restrict__ ex_w) {
    pdl_wait();
    pdl_launch_dependents();
    constexpr bool REPLAY = BWD || WEX;  // phase 3 replays every actor interval the ray reached
    __shared__ float4 s_rec[2][CT_THREADS][4];
    __shared__ float4 s_nv[NRM ? 2 : 1][NRM ? CT_THREADS : 1];  // voxel normals of the staged records
    __shared__ uint32_t s_r[2][CT_THREADS];
    __shared__ uint8_t s_m[2][CT_THREADS];
    __shared__ uint32_t s_sub[DV_MAX_OCTREES + 1];  // sub-list of octree o: [s_sub[o], s_sub[o+1])
    __shared__ uint32_t s_vs[DV_MAX_OCTREES + 1];   // first record of octree o in this view
    constexpr bool ACT = NTA > 0;
    // the backward carries the residual form: the actor partials, the states recorded at actor
    // entries and the replays hold (R, T) instead of the prefix colour, depth (and normal)
    constexpr bool RFORM = BWD;
    __shared__ bool s_flag[ACT ? DV_MAX_OCTREES : 1];  // actor o's box covers this tile
    __shared__ int16_t s_act[ACT ? DV_MAX_OCTREES : 1];
    __shared__ float s_iv[ACT ? NTA : 1][2][ACT ? CT_THREADS : 1];
    __shared__ float s_st[ACT ? NTA : 1][NRM ? 9 : 6][ACT ? CT_THREADS : 1];
    __shared__ int s_nact;

    const int tid = threadIdx.x;
    const int gtile = (int)__ldg(tile_order + (blockIdx.x >> 1));
    const int half = blockIdx.x & 1;
    int view = 0;
    {
        int lo = 0, hi = bp.n_view - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bp.tile_base[mid] <= gtile)
                lo = mid;
            else
                hi = mid - 1;
        }
        view = lo;
    }
    const ViewParams& fp = bp.views[view];
    const OctParams* __restrict__ vo = bp.octs + view * bp.n_oct;
    const int n_oct = bp.n_oct;
    const int tiles_x = fp.tiles_x, W = fp.W, H = fp.H;
    const float t_near = fp.near_, t_far = fp.far_;
    const int tile = gtile - bp.tile_base[view];
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    // the tile's slice of the pair list, kept inside [0, n_pairs] whatever the range words hold (they
    // are only inconsistent after a sort wait that timed out, which the call then reports)
    uint2 rg = __ldg(tile_range + gtile);
    rg.y = (uint32_t)min((int64_t)rg.y, bp.n_pairs);
    rg.x = min(rg.x, rg.y);
    // per-pixel set-up first: its loads overlap the tile set-up below
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t wbit = 1u << ((half * 2 + (warp >> 1)) * 2 + (warp & 1));  // this warp's 8x4 block
    const int u = tx * DV_TILE + (warp & 1) * 8 + (lane & 7);
    const int v = ty * DV_TILE + half * 8 + (warp >> 1) * 4 + (lane >> 3);
    const bool valid = u < W && v < H;
    const int64_t lpix = (int64_t)v * W + u;       // pixel within the view's own images
    const int64_t pix = fp.pix_base + lpix;        // pixel within the call's per-pixel arrays

    float dc[3];
    {
        const float x = ((float)u + 0.5f - fp.cx) / fp.fx;
        const float y = ((float)v + 0.5f - fp.cy) / fp.fy;
        const float in = rsqrtf(fmaf(x, x, fmaf(y, y, 1.0f)));
        dc[0] = x * in;
        dc[1] = y * in;
        dc[2] = in;
    }
    const OctParams& B = vo[0];
    float db_[3];
    rotate(B.A, dc, db_);
    const InvDir ib = inv_dir(db_);

    Pix<NRM> ps;
    ps.C0 = ps.C1 = ps.C2 = ps.D = 0.0f;
    if constexpr (NRM) ps.N0 = ps.N1 = ps.N2 = 0.0f;
    ps.T = 1.0f;
    ps.R = 0.0f;
    ps.n = 0;
    ps.tests = 0;
    ps.boxes = 0;
    ps.done = !valid;
    ExportSink ex;
    ex.n = ex.lim = 0;
    if (WEX) {
        ex.vid = ex_vid;
        ex.w = ex_w;
        ex.sorted_g = bp.sorted_g;
        ex.voff = (int64_t)view * bp.n_vox;
        ex.base = valid ? ex_off[pix] : 0;
        ex.lim = valid ? (uint32_t)(ex_off[pix + 1] - ex.base) : 0u;
    }
    Bwd<NRM> bw;
    if (BWD && valid) {
        bw.g0 = g_rgb ? g_rgb[pix * 3 + 0] : 0.0f;
        bw.g1 = g_rgb ? g_rgb[pix * 3 + 1] : 0.0f;
        bw.g2 = g_rgb ? g_rgb[pix * 3 + 2] : 0.0f;
        bw.gD = g_depth ? g_depth[pix] : 0.0f;
        bw.gA = g_alpha ? g_alpha[pix] : 0.0f;
        bw.Cf0 = fp.rgb[lpix * 3 + 0];
        bw.Cf1 = fp.rgb[lpix * 3 + 1];
        bw.Cf2 = fp.rgb[lpix * 3 + 2];
        bw.Df = fp.depth[lpix];
        bw.Tend = t_final[pix];
    } else {
        bw.g0 = bw.g1 = bw.g2 = bw.gD = bw.gA = 0.0f;
        bw.Cf0 = bw.Cf1 = bw.Cf2 = bw.Df = bw.Tend = 0.0f;
    }
    if constexpr (NRM) {
        bw.gN0 = bw.gN1 = bw.gN2 = bw.Nf0 = bw.Nf1 = bw.Nf2 = 0.0f;
        if (BWD && valid) {
            bw.gN0 = g_normal[pix * 3 + 0];
            bw.gN1 = g_normal[pix * 3 + 1];
            bw.gN2 = g_normal[pix * 3 + 2];
            bw.Nf0 = fp.normal[lpix * 3 + 0];
            bw.Nf1 = fp.normal[lpix * 3 + 1];
            bw.Nf2 = fp.normal[lpix * 3 + 2];
        }
    }
    bw.base = bw.gA * bw.Tend - fmaf(bw.g0, bw.Cf0, fmaf(bw.g1, bw.Cf1, fmaf(bw.g2, bw.Cf2, bw.gD * bw.Df)));
    if constexpr (NRM) bw.base -= fmaf(bw.gN0, bw.Nf0, fmaf(bw.gN1, bw.Nf1, bw.gN2 * bw.Nf2));
    // tile set-up, all loads independent of one another: the view's octree boundaries in
    // the record order, and which actor boxes cover this tile
    for (int i = tid; i <= n_oct; i += CT_THREADS) {
        s_vs[i] = __ldg(vis_start + view * n_oct + i);
        s_sub[i] = rg.x;  // every sub-list start stays inside the tile's slice
    }
    if (ACT) {
        for (int o = tid; o < n_oct; o += CT_THREADS) {
            const OctParams& P = vo[o];
            s_flag[ACT ? o : 0] = o > 0 && P.role == DV_ROLE_ACTOR && P.rect[0] <= tx && tx <= P.rect[2] &&
                                  P.rect[1] <= ty && ty <= P.rect[3];
        }
    }
    __syncthreads();
    // the tile's list is grouped by octree (records are in depth-key order, octree above
    // the BSP path), so octree o's sub-list starts at the first entry whose record is at
    // or after s_vs[o]; entry q finds its octree by a search of s_vs and marks the starts
    // of the octrees between its predecessor's and its own
    {
        auto oct_of = [&](uint32_t r) {
            int lo = 0, hi = n_oct - 1;  // largest o with s_vs[o] <= r
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_vs[mid] <= r)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            return lo;
        };
        for (uint32_t base = rg.x; base < rg.y; base += CT_THREADS) {
            const uint32_t q = base + tid;
            if (q < rg.y) {
                const int o = oct_of(rec_index(bp, pval, q));
                const int op = q > rg.x ? oct_of(rec_index(bp, pval, q - 1)) : -1;
                for (int x = op + 1; x <= o; ++x) s_sub[x] = q;
                if (q + 1 == rg.y)
                    for (int x = o + 1; x <= n_oct; ++x) s_sub[x] = rg.y;
            }
        }
    }
    if (ACT && tid < 32) {
        // actor list of the tile in octree order (warp 0, ballot compaction)
        int n = 0;
        for (int o0 = 0; o0 < n_oct; o0 += 32) {
            const int o = o0 + tid;
            const bool f = o < n_oct && s_flag[ACT ? o : 0];
            const unsigned b = __ballot_sync(0xffffffffu, f);
            if (f) s_act[ACT ? n + __popc(b & ((1u << tid) - 1u)) : 0] = (int16_t)o;
            n += __popc(b);
        }
        if (tid == 0) s_nact = n;
    }
    __syncthreads();

    const int n_ta = ACT ? s_nact : 0;  // 0 at compile time without actors: the actor code folds away
    const int n_lock = n_ta < NTA ? n_ta : NTA;

    // ---- owned actor intervals of this ray (lockstep slots) ----
    for (int q = 0; q < n_lock; ++q) {
        s_iv[q][0][tid] = INFINITY;
        s_iv[q][1][tid] = -INFINITY;
        s_st[q][5][tid] = 0.0f;
    }
    if (valid && n_ta > 0) {
        float tau = t_near;
        for (int guard = 0; guard < n_ta; ++guard) {
            const ActInt it = next_interval(vo, t_near, t_far, s_act, n_ta, dc, tau);
            ps.boxes += n_ta;
            if (it.o < 0) break;
            if (it.q < NTA) {
                s_iv[it.q][0][tid] = it.a;
                s_iv[it.q][1][tid] = it.b;
            }
            tau = it.b;
        }
    }

    // Every sub-list (an actor's, then the background's) streams through the shared
    // two-slot ring, CT_THREADS records per batch (cp.async, one batch ahead).  Each warp
    // visits the records of a batch that touch its 8x4 block (ballot over the pair
    // masks), 32 at a time: chunk(slot, c0, m) gets the ring slot, the first record of
    // the 32 and the mask of those to visit, and returns true once the warp has nothing
    // left to do in this list.  The batch loop, its barriers and its early exit are
    // CTA-uniform.
    auto stream = [&](uint32_t q0, uint32_t q1, auto&& chunk) {
        const uint32_t n_batch = q1 > q0 ? (q1 - q0 + CT_THREADS - 1) / CT_THREADS : 0u;
        uint32_t r_ahead = 0, m_ahead = 0;
        if (n_batch > 0) {
            const uint32_t qa = q0 + tid;
            if (qa < q1) {
                const uint32_t r = rec_index(bp, pval, qa);
                const float4* R = rec[r].v;
#pragma unroll
                for (int k = 0; k < 4; ++k) cp_async16(&s_rec[0][tid][k], R + k);
                if (NRM) cp_async16(&s_nv[0][NRM ? tid : 0], bp.nrm + r);
                s_r[0][tid] = r;
                s_m[0][tid] = __ldg(pmask + qa);
            }
            cp_async_commit();
            const uint32_t qb = q0 + CT_THREADS + tid;
            if (qb < q1) {
                r_ahead = rec_index(bp, pval, qb);
                m_ahead = __ldg(pmask + qb);
            }
        }
        bool fin = false;
        for (uint32_t bi = 0; bi < n_batch; ++bi) {
            const int slot = bi & 1;
            {
                const uint32_t qa = q0 + (bi + 1) * CT_THREADS + tid;
                if (qa < q1) {
                    const float4* R = rec[r_ahead].v;
#pragma unroll
                    for (int k = 0; k < 4; ++k) cp_async16(&s_rec[slot ^ 1][tid][k], R + k);
                    if (NRM) cp_async16(&s_nv[NRM ? (slot ^ 1) : 0][NRM ? tid : 0], bp.nrm + r_ahead);
                    s_r[slot ^ 1][tid] = r_ahead;
                    s_m[slot ^ 1][tid] = (uint8_t)m_ahead;
                }
                cp_async_commit();
                const uint32_t qb = q0 + (bi + 2) * CT_THREADS + tid;
                if (qb < q1) {
                    r_ahead = rec_index(bp, pval, qb);
                    m_ahead = __ldg(pmask + qb);
                }
            }
            cp_async_wait_one();  // batch bi has landed (only batch bi+1 may still be in flight)
            __syncthreads();
            const uint32_t cnt = min((uint32_t)CT_THREADS, q1 - q0 - bi * CT_THREADS);
            for (uint32_t c0 = 0; c0 < cnt && !fin; c0 += 32) {
                const uint32_t jl = c0 + lane;
                const unsigned m = __ballot_sync(0xffffffffu, jl < cnt && (s_m[slot][jl < cnt ? jl : 0] & wbit));
                fin = chunk(slot, c0, m);
            }
            // every warp is done with this slot before batch bi+2 is copied into it
            if (__syncthreads_or(!fin) == 0) break;
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy outlives the list (early exit)
        __syncthreads();                                     // the ring is free for the next list
    };

    // voxel normal of staged record j (zero without normals)
    auto staged_nv = [&](int slot, uint32_t j) {
        return NRM ? s_nv[NRM ? slot : 0][NRM ? j : 0] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    };
    constexpr int NV = GradLayout<NRM>::NV;
    constexpr int GS = GradLayout<NRM>::STRIDE;

    // Lockstep walk of actor o's sub-list: lanes not yet done composite the segments inside
    // their interval [a, b] of that actor into pt, with the stop rule (and, with G, the
    // per-record gradients reduced across the warp).
    auto walk_actor = [&](Pix<NRM>& pt, int o, float a, float b, auto grad, auto wex) {
        constexpr bool G = decltype(grad)::value;
        constexpr bool X = decltype(wex)::value;
        const OctParams& P = vo[o];
        float d[3];
        rotate(P.A, dc, d);
        const InvDir inv = inv_dir(d);
        stream(s_sub[o], s_sub[o + 1], [&](int slot, uint32_t c0, unsigned m) -> bool {
            while (m) {
                if (__all_sync(0xffffffffu, pt.done)) return true;
                const uint32_t j = c0 + (uint32_t)(__ffs(m) - 1);
                m &= m - 1;
                if constexpr (!G && !X && KS == 1) {
                    if (m) {
                        // two records at once (no gradients): both slab tests and optical depths, then the
                        // two compositing steps in list order with the stop rule -- the arithmetic of two
                        // single steps, with more independent work per warp on the actor walks
                        const uint32_t j1 = c0 + (uint32_t)(__ffs(m) - 1);
                        m &= m - 1;
                        const float4 g0 = s_rec[slot][j][0], g1 = s_rec[slot][j1][0];
                        float u0, v0, u1, v1;
                        const bool x0 = slab_cube(inv, g0, u0, v0), x1 = slab_cube(inv, g1, u1, v1);
                        u0 = fmaxf(u0, a);
                        v0 = fminf(v0, b);
                        u1 = fmaxf(u1, a);
                        v1 = fminf(v1, b);
                        const bool live = !pt.done;
                        const bool h0 = live && x0 && v0 > u0, h1 = live && x1 && v1 > u1;
                        const float s0 = h0 ? u0 : 0.0f, e0 = h0 ? v0 : 0.0f, s1 = h1 ? u1 : 0.0f, e1 = h1 ? v1 : 0.0f;
                        const float4 col0 = s_rec[slot][j][3], col1 = s_rec[slot][j1][3];
                        const float r0[3] = {g0.x, g0.y, g0.z}, r1[3] = {g1.x, g1.y, g1.z};
                        const float tau0 = seg_tau<false, 1>(s_rec[slot][j][1], s_rec[slot][j][2], col0.w, r0, d, s0,
                                                             e0, bp.K, bp.inv_k, bp.activation, nullptr, nullptr);
                        const float tau1 = seg_tau<false, 1>(s_rec[slot][j1][1], s_rec[slot][j1][2], col1.w, r1, d, s1,
                                                             e1, bp.K, bp.inv_k, bp.activation, nullptr, nullptr);
                        auto apply = [&](float tau, float4 col, float4 nv, float t0, float t1) {
                            if constexpr (RFORM) {
                                const float ee = __expf(-tau);
                                const float w = pt.T * (1.0f - ee);
                                const float mid = 0.5f * (t0 + t1);
                                float sg = fmaf(bw.g0, col.x, fmaf(bw.g1, col.y, fmaf(bw.g2, col.z, bw.gD * mid)));
                                if constexpr (NRM) sg = fmaf(bw.gN0, nv.x, fmaf(bw.gN1, nv.y, fmaf(bw.gN2, nv.z, sg)));
                                pt.R = fmaf(w, sg, pt.R);
                                pt.T = pt.T * ee;
                                pt.n += 1;
                                if (pt.T < bp.eps_stop) pt.done = true;
                            } else {
                                composite_tau<NRM>(pt, tau, col, nv, t0, t1, bp.eps_stop);
                            }
                        };
                        pt.tests += live ? 1u : 0u;
                        if (h0) apply(tau0, col0, staged_nv(slot, j), s0, e0);
                        pt.tests += (live && !pt.done) ? 1u : 0u;
                        if (h1 && !pt.done) apply(tau1, col1, staged_nv(slot, j1), s1, e1);
                        continue;
                    }
                }
                if constexpr (G && RFORM && !X && KS == 1) {
                    // replay with gradients: inside one actor interval a lane meets a record at most once
                    const float4 g = s_rec[slot][j][0];
                    const bool live = !pt.done;
                    float t0, t1;
                    const bool xs = slab_cube(inv, g, t0, t1);
                    t0 = fmaxf(t0, a);
                    t1 = fminf(t1, b);
                    const bool hit = live && xs && t1 > t0;
                    pt.tests += live ? 1u : 0u;
                    if (!__any_sync(0xffffffffu, hit)) continue;
                    float acc[NV];
                    bwd_single_step<NRM>(pt, bw, bp, g, s_rec[slot][j][1], s_rec[slot][j][2], s_rec[slot][j][3],
                                         staged_nv(slot, j), d, hit ? t0 : 0.0f, hit ? t1 : 0.0f, hit, acc);
                    warp_reduce_add<NV>(acc, grad_rec + (size_t)s_r[slot][j] * GS);
                    continue;
                }
                float acc[NV];
                if (G) {
#pragma unroll
                    for (int i = 0; i < NV; ++i) acc[i] = 0.0f;
                }
                bool hit = false;
                if (!pt.done) {
                    pt.tests += 1;
                    const float4 g = s_rec[slot][j][0];
                    float t0, t1;
                    if (slab_cube(inv, g, t0, t1)) {
                        t0 = fmaxf(t0, a);
                        t1 = fminf(t1, b);
                        if (t1 > t0) {
                            const float rel[3] = {g.x, g.y, g.z};
                            add_segment<G, true, KS, NRM, X, RFORM>(pt, bw, bp, s_rec[slot][j][1], s_rec[slot][j][2],
                                                             s_rec[slot][j][3], staged_nv(slot, j), rel, d, t0, t1,
                                                             acc, s_r[slot][j], &ex);
                            hit = true;
                        }
                    }
                }
                if (G) {
                    const unsigned any = __ballot_sync(0xffffffffu, hit);
                    if (any) warp_reduce_add<NV>(acc, grad_rec + (size_t)s_r[slot][j] * GS);
                }
            }
            return __all_sync(0xffffffffu, pt.done);
        });
    };

    // ---- phase 1: partial composite of every lockstep actor interval ----
    for (int q = 0; q < n_lock; ++q) {
        const float a = s_iv[q][0][tid], b = s_iv[q][1][tid];
        const bool act = valid && b > a;
        if (__syncthreads_or(act) == 0) continue;
        Pix<NRM> pt;
        pt.C0 = pt.C1 = pt.C2 = pt.D = 0.0f;
        if constexpr (NRM) pt.N0 = pt.N1 = pt.N2 = 0.0f;
        pt.T = 1.0f;
        pt.R = 0.0f;
        pt.n = 0;
        pt.tests = 0;
        pt.boxes = 0;
        pt.done = !act;
        // a lane whose own transmittance already falls below eps_stop will stop inside this
        // actor whatever T it enters with (T <= 1), so its partial may stop there too
        walk_actor(pt, s_act[q], a, b, std::false_type(), std::false_type());
        ps.tests += pt.tests;
        if (act && RFORM) {
            s_st[q][0][tid] = pt.R;
            s_st[q][4][tid] = pt.T;
            s_st[q][5][tid] = __int_as_float((int)pt.n);
        } else if (act) {
            s_st[q][0][tid] = pt.C0;
            s_st[q][1][tid] = pt.C1;
            s_st[q][2][tid] = pt.C2;
            s_st[q][3][tid] = pt.D;
            s_st[q][4][tid] = pt.T;
            s_st[q][5][tid] = __int_as_float((int)pt.n);
            if constexpr (NRM) {
                s_st[q][NRM ? 6 : 0][tid] = pt.N0;
                s_st[q][NRM ? 7 : 0][tid] = pt.N1;
                s_st[q][NRM ? 8 : 0][tid] = pt.N2;
            }
        }
    }

    // ---- phase 2: background walk, applying actor partials in order ----
    float tau_cur = t_near;
    ActInt nxt;
    nxt.o = -1;
    if (valid && n_ta > 0) {
        nxt = next_interval(vo, t_near, t_far, s_act, n_ta, dc, tau_cur);
        ps.boxes += n_ta;
    }
    // enters actor interval `it`: apply its partial, or stop inside it, or walk it per lane
    auto enter_actor = [&](const ActInt& it) {
        if (RFORM && it.q < NTA) {
            // backward: record the entry state (R, T) for the replay, then apply the partial
            const int q = it.q;
            const float pR = s_st[q][0][tid], pT = s_st[q][4][tid];
            const uint32_t pn = (uint32_t)__float_as_int(s_st[q][5][tid]);
            const bool stop_inside = ps.T * pT < bp.eps_stop;
            s_st[q][0][tid] = ps.R;
            s_st[q][4][tid] = ps.T;
            s_st[q][5][tid] = stop_inside ? 2.0f : 1.0f;
            if (stop_inside) {
                ps.done = true;
            } else {
                ps.R = fmaf(ps.T, pR, ps.R);
                ps.T = ps.T * pT;
                ps.n += pn;
            }
        } else if (it.q < NTA) {
            const int q = it.q;
            const float pC0 = s_st[q][0][tid], pC1 = s_st[q][1][tid], pC2 = s_st[q][2][tid];
            const float pD = s_st[q][3][tid], pT = s_st[q][4][tid];
            const uint32_t pn = (uint32_t)__float_as_int(s_st[q][5][tid]);
            float pN0 = 0.0f, pN1 = 0.0f, pN2 = 0.0f;
            if (NRM) {
                pN0 = s_st[q][NRM ? 6 : 0][tid];
                pN1 = s_st[q][NRM ? 7 : 0][tid];
                pN2 = s_st[q][NRM ? 8 : 0][tid];
            }
            const bool stop_inside = ps.T * pT < bp.eps_stop;
            if (REPLAY || stop_inside) {
                s_st[q][0][tid] = ps.C0;
                s_st[q][1][tid] = ps.C1;
                s_st[q][2][tid] = ps.C2;
                s_st[q][3][tid] = ps.D;
                s_st[q][4][tid] = ps.T;
                if constexpr (NRM) {
                    s_st[q][NRM ? 6 : 0][tid] = ps.N0;
                    s_st[q][NRM ? 7 : 0][tid] = ps.N1;
                    s_st[q][NRM ? 8 : 0][tid] = ps.N2;
                }
            }
            s_st[q][5][tid] = stop_inside ? 2.0f : 1.0f;
            if (stop_inside) {
                ps.done = true;
            } else {
                ps.C0 = fmaf(ps.T, pC0, ps.C0);
                ps.C1 = fmaf(ps.T, pC1, ps.C1);
                ps.C2 = fmaf(ps.T, pC2, ps.C2);
                ps.D = fmaf(ps.T, pD, ps.D);
                if constexpr (NRM) {
                    ps.N0 = fmaf(ps.T, pN0, ps.N0);
                    ps.N1 = fmaf(ps.T, pN1, ps.N1);
                    ps.N2 = fmaf(ps.T, pN2, ps.N2);
                }
                ps.T = ps.T * pT;
                ps.n += pn;
            }
        } else {
            // the out-of-line walk takes copies: an object whose address reaches a call stays in
            // local memory everywhere, so the hot-path state (ps, bw, dc, nxt, ex) never does
            Pix<NRM> pl = ps;
            const Bwd<NRM> bl = bw;
            const ActInt il = it;
            const float dl[3] = {dc[0], dc[1], dc[2]};
            ExportSink xl = ex;
            walk_actor_lane<BWD, KS, NRM, WEX>(pl, bl, bp, vo, il, pval, pmask, wbit, rec, s_sub[il.o],
                                               s_sub[il.o + 1], dl, grad_rec, &xl);
            ps = pl;
            ex = xl;
        }
    };

    stream(s_sub[0], s_sub[1], [&](int slot, uint32_t c0, unsigned m) -> bool {
        // one record of the batch, visited by the whole warp: actor entries, stop rule, gradients
        auto visit = [&](uint32_t j) {
            if constexpr (BWD && NTA == 0 && KS == 1) {
                // plain tiles, one sample per segment: a lane meets a record at most once, so once any lane
                // of the warp hits it every lane runs the same arithmetic without branches, a lane that
                // misses (or is done) on the empty segment [0, 0], whose optical depth, weight and gradient
                // are exactly zero; the gradient values are written, not accumulated, so nothing is cleared
                const float4 g = s_rec[slot][j][0];
                const bool live = !ps.done;
                float t_in, t_out;
                const bool xs = slab_cube(ib, g, t_in, t_out);
                t_in = fmaxf(fmaxf(t_in, t_near), tau_cur);
                t_out = fminf(t_out, t_far);
                const bool hit = live && xs && t_out > t_in;
                ps.tests += live ? 1u : 0u;
                if (!__any_sync(0xffffffffu, hit)) return;
                const float u0 = hit ? t_in : 0.0f, u1 = hit ? t_out : 0.0f;
                float acc[NV];
                bwd_single_step<NRM>(ps, bw, bp, g, s_rec[slot][j][1], s_rec[slot][j][2], s_rec[slot][j][3],
                                     staged_nv(slot, j), db_, u0, u1, hit, acc);
                warp_reduce_add<NV>(acc, grad_rec + (size_t)s_r[slot][j] * GS);
                return;
            }
            if constexpr (BWD && NTA > 0 && KS == 1) {
                // actor tiles: a background record that no lane's segment carries into the next actor
                // interval is met at most once by every lane, so it takes the same branch-free step; a
                // record some lane crosses an actor entry in goes through the general path below
                const float4 g = s_rec[slot][j][0];
                const bool live = !ps.done;
                float t_in, t_out;
                const bool xs = slab_cube(ib, g, t_in, t_out);
                t_in = fmaxf(t_in, t_near);
                t_out = fminf(t_out, t_far);
                const bool in = live && xs && t_out > t_in;
                if (!__any_sync(0xffffffffu, in && nxt.o >= 0 && nxt.a < t_out)) {
                    const float cur = fmaxf(t_in, tau_cur);
                    const bool hit = in && t_out > cur;
                    ps.tests += live ? 1u : 0u;
                    if (!__any_sync(0xffffffffu, hit)) return;
                    float acc[NV];
                    bwd_single_step<NRM>(ps, bw, bp, g, s_rec[slot][j][1], s_rec[slot][j][2], s_rec[slot][j][3],
                                         staged_nv(slot, j), db_, hit ? cur : 0.0f, hit ? t_out : 0.0f, hit, acc);
                    warp_reduce_add<NV>(acc, grad_rec + (size_t)s_r[slot][j] * GS);
                    return;
                }
            }
            float acc[NV];
            if (BWD) {
#pragma unroll
                for (int i = 0; i < NV; ++i) acc[i] = 0.0f;
            }
            bool contributed = false;
            const float4 g = s_rec[slot][j][0];
            float t_in, t_out;
            const float rel[3] = {g.x, g.y, g.z};
            if (!ps.done) ps.tests += 1;
            if (!ps.done && slab_cube(ib, g, t_in, t_out)) {
                t_in = fmaxf(t_in, t_near);
                t_out = fminf(t_out, t_far);
                if (t_out > t_in) {
                    const float4 da = s_rec[slot][j][1], dd = s_rec[slot][j][2], col = s_rec[slot][j][3];
                    const float4 nv = staged_nv(slot, j);
                    float cur = fmaxf(t_in, tau_cur);
                    while (nxt.o >= 0 && nxt.a < t_out && !ps.done) {
                        if (nxt.a > cur) {
                            add_segment<BWD, true, KS, NRM, WEX, RFORM>(ps, bw, bp, da, dd, col, nv, rel, db_, cur, nxt.a,
                                                                 acc, s_r[slot][j], &ex);
                            contributed = true;
                            if (ps.done) break;
                        }
                        enter_actor(nxt);
                        tau_cur = nxt.b;
                        cur = fmaxf(cur, nxt.b);
                        nxt = next_interval(vo, t_near, t_far, s_act, n_ta, dc, tau_cur);
                        ps.boxes += n_ta;
                    }
                    if (!ps.done && t_out > cur) {
                        add_segment<BWD, true, KS, NRM, WEX, RFORM>(ps, bw, bp, da, dd, col, nv, rel, db_, cur, t_out, acc,
                                                             s_r[slot][j], &ex);
                        contributed = true;
                    }
                }
            }
            if (BWD) {
                // every lane visits record j of the batch together: reduce across the warp
                const unsigned any = __ballot_sync(0xffffffffu, contributed);
                if (any) warp_reduce_add<NV>(acc, grad_rec + (size_t)s_r[slot][j] * GS);
            }
        };
        bool warp_done = false;
        while (m) {
            if (__all_sync(0xffffffffu, ps.done)) {
                warp_done = true;
                break;
            }
            const uint32_t j0 = c0 + (uint32_t)(__ffs(m) - 1);
            m &= m - 1;
            if (REPLAY || m == 0) {
                visit(j0);
                continue;
            }
            const uint32_t j1 = c0 + (uint32_t)(__ffs(m) - 1);
            m &= m - 1;
            // forward, two records at once: both slab tests, then (unless a lane enters an
            // actor interval inside either segment) both optical depths, then compositing in
            // list order with the stop rule -- the same arithmetic as two visits
            const float4 g0 = s_rec[slot][j0][0], g1 = s_rec[slot][j1][0];
            float a0, b0, a1, b1;
            const bool x0 = slab_cube(ib, g0, a0, b0);
            const bool x1 = slab_cube(ib, g1, a1, b1);
            a0 = fmaxf(a0, t_near);
            b0 = fminf(b0, t_far);
            a1 = fmaxf(a1, t_near);
            b1 = fminf(b1, t_far);
            const bool live = !ps.done;
            const bool in0 = live && x0 && b0 > a0, in1 = live && x1 && b1 > a1;
            const bool cross = nxt.o >= 0 && ((in0 && nxt.a < b0) || (in1 && nxt.a < b1));
            if (__any_sync(0xffffffffu, cross)) {
                visit(j0);
                visit(j1);
                continue;
            }
            a0 = fmaxf(a0, tau_cur);
            a1 = fmaxf(a1, tau_cur);
            const bool h0 = in0 && b0 > a0, h1 = in1 && b1 > a1;
            const float4 da0 = s_rec[slot][j0][1], dd0 = s_rec[slot][j0][2], col0 = s_rec[slot][j0][3];
            const float4 da1 = s_rec[slot][j1][1], dd1 = s_rec[slot][j1][2], col1 = s_rec[slot][j1][3];
            const float r0[3] = {g0.x, g0.y, g0.z}, r1[3] = {g1.x, g1.y, g1.z};
            const float u0 = h0 ? a0 : 0.0f, v0 = h0 ? b0 : 0.0f, u1 = h1 ? a1 : 0.0f, v1 = h1 ? b1 : 0.0f;
            const float tau0 = seg_tau<false, KS>(da0, dd0, col0.w, r0, db_, u0, v0, bp.K, bp.inv_k, bp.activation,
                                                  nullptr, nullptr);
            const float tau1 = seg_tau<false, KS>(da1, dd1, col1.w, r1, db_, u1, v1, bp.K, bp.inv_k, bp.activation,
                                                  nullptr, nullptr);
            ps.tests += live ? 1u : 0u;
            if (h0) composite_tau<NRM>(ps, tau0, col0, staged_nv(slot, j0), u0, v0, bp.eps_stop);
            ps.tests += (live && !ps.done) ? 1u : 0u;
            if (h1 && !ps.done) composite_tau<NRM>(ps, tau1, col1, staged_nv(slot, j1), u1, v1, bp.eps_stop);
        }
        return warp_done || __all_sync(0xffffffffu, ps.done);
    });
    // actor intervals behind the last background hit
    while (nxt.o >= 0 && !ps.done) {
        enter_actor(nxt);
        tau_cur = nxt.b;
        nxt = next_interval(vo, t_near, t_far, s_act, n_ta, dc, tau_cur);
        ps.boxes += n_ta;
    }

    // ---- phase 3: actor intervals replayed from their entry state ----
    //   forward: only those where the ray stops; backward: every one reached (gradients)
    for (int q = 0; q < n_lock; ++q) {
        const int status = valid ? (int)s_st[q][5][tid] : 0;
        const bool act = REPLAY ? status >= 1 : status == 2;
        if (__syncthreads_or(act) == 0) continue;
        Pix<NRM> pt;
        pt.T = act ? s_st[q][4][tid] : 1.0f;
        if (RFORM) {
            pt.R = act ? s_st[q][0][tid] : 0.0f;
            pt.C0 = pt.C1 = pt.C2 = pt.D = 0.0f;
            if constexpr (NRM) pt.N0 = pt.N1 = pt.N2 = 0.0f;
        } else {
            pt.R = 0.0f;
            pt.C0 = act ? s_st[q][0][tid] : 0.0f;
            pt.C1 = act ? s_st[q][1][tid] : 0.0f;
            pt.C2 = act ? s_st[q][2][tid] : 0.0f;
            pt.D = act ? s_st[q][3][tid] : 0.0f;
            if constexpr (NRM) {
                pt.N0 = act ? s_st[q][6][tid] : 0.0f;
                pt.N1 = act ? s_st[q][7][tid] : 0.0f;
                pt.N2 = act ? s_st[q][8][tid] : 0.0f;
            }
        }
        pt.n = 0;
        pt.tests = 0;
        pt.boxes = 0;
        pt.done = !act;
        walk_actor(pt, s_act[q], s_iv[q][0][tid], s_iv[q][1][tid], std::integral_constant<bool, BWD>(),
                   std::integral_constant<bool, WEX>());
        ps.tests += pt.tests;
        if (!REPLAY && act) {
            ps.C0 = pt.C0;
            ps.C1 = pt.C1;
            ps.C2 = pt.C2;
            ps.D = pt.D;
            if constexpr (NRM) {
                ps.N0 = pt.N0;
                ps.N1 = pt.N1;
                ps.N2 = pt.N2;
            }
            ps.T = pt.T;
            ps.n += pt.n;
        }
    }

    if (!REPLAY && work) {
        unsigned long long t = ps.tests, b = ps.boxes, n = ps.n;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            t += __shfl_down_sync(0xffffffffu, t, off);
            b += __shfl_down_sync(0xffffffffu, b, off);
            n += __shfl_down_sync(0xffffffffu, n, off);
        }
        if (lane == 0) {
            atomicAdd(work + 0, t);
            atomicAdd(work + 1, b);
            atomicAdd(work + 2, n);
        }
    }
    if (!REPLAY && valid) {
        fp.rgb[lpix * 3 + 0] = ps.C0;
        fp.rgb[lpix * 3 + 1] = ps.C1;
        fp.rgb[lpix * 3 + 2] = ps.C2;
        fp.depth[lpix] = ps.D;
        fp.alpha[lpix] = 1.0f - ps.T;
        n_seg[pix] = ps.n;
        t_final[pix] = ps.T;
        if constexpr (NRM) {
            fp.normal[lpix * 3 + 0] = ps.N0;
            fp.normal[lpix * 3 + 1] = ps.N1;
            fp.normal[lpix * 3 + 2] = ps.N2;
        }
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

struct ShBwdParams {
    BatchParams bp;
    float* d_dens[DV_MAX_OCTREES];
    float* d_sh[DV_MAX_OCTREES];
};

template <bool NRM>
__global__ void __launch_bounds__(256) k_sh_bwd(const __grid_constant__ ShBwdParams sp,
                                                const uint32_t* __restrict__ sorted_g, int64_t n_vis,
                                                const VoxRec* __restrict__ rec, const float* __restrict__ grad_rec) {
    pdl_wait();
    pdl_launch_dependents();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_vis) return;
    const BatchParams& bp = sp.bp;
    const uint32_t gidx = sorted_g[r];
    const int view = (int)(gidx / (uint64_t)bp.n_vox);
    const int64_t gv = (int64_t)gidx - (int64_t)view * bp.n_vox;
    int lo = 0, hi = bp.n_oct - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bp.vox_offset[mid] <= gv)
            lo = mid;
        else
            hi = mid - 1;
    }
    const OctParams& P = bp.octs[view * bp.n_oct + lo];
    const int64_t v = gv - bp.vox_offset[lo];
    const float* gr = grad_rec + (size_t)r * GradLayout<NRM>::STRIDE;
    float* d_dens = sp.d_dens[lo];
    float* d_sh = sp.d_sh[lo];
    // several views may touch the same voxel: accumulate with atomics (16-byte vector
    // atomics where the caller's rows are 16-byte aligned)
    float4 g03 = *reinterpret_cast<const float4*>(gr), g47 = *reinterpret_cast<const float4*>(gr + 4);
    if (NRM) {
        // through the voxel normal n_w = R n_l, n_l = -g / |g| with g the corner-difference
        // gradient (as in the records kernel): dL/dg = -(dL/dn_l - n_l (n_l . dL/dn_l)) / |g|,
        // and each corner enters g_a with sign + on the high side of axis a, - on the low side
        const float dw0 = gr[11], dw1 = gr[12], dw2 = gr[13];
        if (d_dens && (dw0 != 0.0f || dw1 != 0.0f || dw2 != 0.0f)) {
            // the raw corner densities, as the records kernel used them for the voxel normal
            const float4* d4 = reinterpret_cast<const float4*>(P.dens + v * 8);
            const float4 da = __ldg(d4), db = __ldg(d4 + 1);
            const float gx = (da.y + da.w + db.y + db.w) - (da.x + da.z + db.x + db.z);
            const float gy = (da.z + da.w + db.z + db.w) - (da.x + da.y + db.x + db.y);
            const float gz = (db.x + db.y + db.z + db.w) - (da.x + da.y + da.z + da.w);
            const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
            if (g2 > 0.0f) {
                const float ig = rsqrtf(g2);
                const float nl[3] = {-gx * ig, -gy * ig, -gz * ig};
                float dn[3];
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    dn[k] = fmaf(P.Rw[0 * 3 + k], dw0, fmaf(P.Rw[1 * 3 + k], dw1, P.Rw[2 * 3 + k] * dw2));
                const float nd = fmaf(nl[0], dn[0], fmaf(nl[1], dn[1], nl[2] * dn[2]));
                const float dgx = -(dn[0] - nl[0] * nd) * ig, dgy = -(dn[1] - nl[1] * nd) * ig,
                            dgz = -(dn[2] - nl[2] * nd) * ig;
                // corner c = (x, y, z) bits: + dg_a where bit a is set, - where clear
                g03.x += -dgx - dgy - dgz;
                g03.y += dgx - dgy - dgz;
                g03.z += -dgx + dgy - dgz;
                g03.w += dgx + dgy - dgz;
                g47.x += -dgx - dgy + dgz;
                g47.y += dgx - dgy + dgz;
                g47.z += -dgx + dgy + dgz;
                g47.w += dgx + dgy + dgz;
            }
        }
    }
    if (d_dens) {
        float* dd = d_dens + v * 8;
        if ((reinterpret_cast<uintptr_t>(dd) & 15) == 0) {
            if (g03.x != 0.0f || g03.y != 0.0f || g03.z != 0.0f || g03.w != 0.0f)
                atomicAdd(reinterpret_cast<float4*>(dd), g03);
            if (g47.x != 0.0f || g47.y != 0.0f || g47.z != 0.0f || g47.w != 0.0f)
                atomicAdd(reinterpret_cast<float4*>(dd) + 1, g47);
        } else {
            const float gd[8] = {g03.x, g03.y, g03.z, g03.w, g47.x, g47.y, g47.z, g47.w};
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (gd[c] != 0.0f) atomicAdd(dd + c, gd[c]);
        }
    }
    // colour channels clamped at zero in the forward (stored clamped in the record) pass no
    // gradient to the SH coefficients
    const float4 col = rec[r].v[3];
    const float m0 = col.x > 0.0f ? gr[8] : 0.0f, m1 = col.y > 0.0f ? gr[9] : 0.0f, m2 = col.z > 0.0f ? gr[10] : 0.0f;
    if (!d_sh || (m0 == 0.0f && m1 == 0.0f && m2 == 0.0f)) return;
    const float4 g = rec[r].v[0];  // (min - camera centre, size): same direction as the records kernel
    float gx = fmaf(0.5f, g.w, g.x);
    float gy = fmaf(0.5f, g.w, g.y);
    float gz = fmaf(0.5f, g.w, g.z);
    const float gl = sqrtf(gx * gx + gy * gy + gz * gz);
    const float ig = gl > 0.0f ? 1.0f / gl : 0.0f;
    gx *= ig;
    gy *= ig;
    gz *= ig;
    float b[16];
    sh_basis_f(P.sh_degree, gx, gy, gz, b);
    const int nsh = (P.sh_degree + 1) * (P.sh_degree + 1);
    float* ds = d_sh + v * nsh * 3;
    if ((nsh * 3) % 4 == 0 && (reinterpret_cast<uintptr_t>(ds) & 15) == 0) {
        // coefficient rows (q, channel) flattened: element e = 3 q + channel
        const float m[3] = {m0, m1, m2};
#pragma unroll
        for (int e0 = 0; e0 < 48; e0 += 4) {
            if (e0 >= nsh * 3) break;
            float x[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = e0 + i;
                x[i] = b[e / 3] * m[e % 3];
            }
            atomicAdd(reinterpret_cast<float4*>(ds + e0), make_float4(x[0], x[1], x[2], x[3]));
        }
    } else {
        for (int q = 0; q < nsh; ++q) {
            if (m0 != 0.0f) atomicAdd(ds + q * 3 + 0, b[q] * m0);
            if (m1 != 0.0f) atomicAdd(ds + q * 3 + 1, b[q] * m1);
            if (m2 != 0.0f) atomicAdd(ds + q * 3 + 2, b[q] * m2);
        }
    }
}

// Three launches per compositing pass, two CTAs per tile, over the three groups of the tile order:
// the tiles that 5 or more actor boxes cover (8 lockstep actor slots), those that 1 to 4 cover (4
// slots), and the others (no actor machinery).  They run side by side: the two actor launches on the
// context's two extra streams (the device's highest priority, so their CTAs -- the heaviest tiles of
// a frame -- are dispatched first), forked from and joined back into the call's stream by events, the
// plain launch on the call's stream.  Without the extra streams they run one after the other.
template <bool BWD, int KS, bool NRM, bool WEX>
void composite_launch(const BatchParams& bp, const VoxRec* rec, const uint32_t* pval, const uint8_t* pmask,
                      const uint2* tile_range, const uint32_t* vis_start, const uint32_t* tile_order,
                      uint32_t* n_seg, float* t_final, const float* g_rgb, const float* g_depth,
                      const float* g_alpha, const float* g_normal, float* grad_rec, unsigned long long* work,
                      const int64_t* ex_off, uint32_t* ex_vid, float* ex_w, const Fork* fk, cudaStream_t s) {
    const int n_large = bp.n_tiles_large, n_small = bp.n_tiles_small;
    const int n_plain = bp.n_tiles - n_large - n_small;
    const int groups = (n_large > 0) + (n_small > 0) + (n_plain > 0);
    const bool fork = fk && fk->side && fk->side2 && groups > 1;
    cudaStream_t s_large = s, s_small = s;
    if (fork && cudaEventRecord(fk->ev_fork, s) == cudaSuccess) {
        if (n_large > 0 && cudaStreamWaitEvent(fk->side, fk->ev_fork, 0) == cudaSuccess) s_large = fk->side;
        if (n_small > 0 && cudaStreamWaitEvent(fk->side2, fk->ev_fork, 0) == cudaSuccess) s_small = fk->side2;
    }
    if (n_large > 0) {
        launch_pdl(k_composite<BWD, KS, NRM, WEX, NTA_LARGE>, dim3(2 * n_large), dim3(CT_THREADS), s_large, bp, rec,
                   pval, pmask, tile_range, vis_start, tile_order, n_seg, t_final, g_rgb, g_depth, g_alpha, g_normal,
                   grad_rec, work, ex_off, ex_vid, ex_w);
        count_launches(1);
    }
    if (n_small > 0) {
        launch_pdl(k_composite<BWD, KS, NRM, WEX, NTA_SMALL>, dim3(2 * n_small), dim3(CT_THREADS), s_small, bp, rec,
                   pval, pmask, tile_range, vis_start, tile_order + n_large, n_seg, t_final, g_rgb, g_depth, g_alpha,
                   g_normal, grad_rec, work, ex_off, ex_vid, ex_w);
        count_launches(1);
    }
    if (n_plain > 0) {
        launch_pdl(k_composite<BWD, KS, NRM, WEX, 0>, dim3(2 * n_plain), dim3(CT_THREADS), s, bp, rec, pval, pmask,
                   tile_range, vis_start, tile_order + n_large + n_small, n_seg, t_final, g_rgb, g_depth, g_alpha,
                   g_normal, grad_rec, work, ex_off, ex_vid, ex_w);
        count_launches(1);
    }
    if (s_large != s) {
        cudaEventRecord(fk->ev_join, s_large);
        cudaStreamWaitEvent(s, fk->ev_join, 0);
    }
    if (s_small != s) {
        cudaEventRecord(fk->ev_join2, s_small);
        cudaStreamWaitEvent(s, fk->ev_join2, 0);
    }
}

template <bool NRM>
void composite_fwd_k(const BatchParams& bp, const VoxRec* rec, const uint32_t* pair_val, const uint8_t* pair_mask,
                     const uint2* tile_range, const uint32_t* vis_start, const uint32_t* tile_order, uint32_t* n_seg,
                     float* t_final, unsigned long long* work, const Fork* fk, cudaStream_t s) {
    if (bp.K == 1)
        composite_launch<false, 1, NRM, false>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, n_seg,
                                               t_final, nullptr, nullptr, nullptr, nullptr, nullptr, work, nullptr,
                                               nullptr, nullptr, fk, s);
    else
        composite_launch<false, 0, NRM, false>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, n_seg,
                                               t_final, nullptr, nullptr, nullptr, nullptr, nullptr, work, nullptr,
                                               nullptr, nullptr, fk, s);
}

template <bool NRM>
void composite_bwd_k(const BatchParams& bp, const VoxRec* rec, const uint32_t* pair_val, const uint8_t* pair_mask,
                     const uint2* tile_range, const uint32_t* vis_start, const uint32_t* tile_order,
                     const float* t_final, const float* g_rgb, const float* g_depth, const float* g_alpha,
                     const float* g_normal, float* grad_rec, const Fork* fk, cudaStream_t s) {
    // the kernel's per-pixel forward results (final T here, C, D, N through the view parameters)
    // are only read in the backward
    float* tf = const_cast<float*>(t_final);
    if (bp.K == 1)
        composite_launch<true, 1, NRM, false>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, nullptr,
                                              tf, g_rgb, g_depth, g_alpha, g_normal, grad_rec, nullptr, nullptr,
                                              nullptr, nullptr, fk, s);
    else
        composite_launch<true, 0, NRM, false>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, nullptr,
                                              tf, g_rgb, g_depth, g_alpha, g_normal, grad_rec, nullptr, nullptr,
                                              nullptr, nullptr, fk, s);
}

}  // namespace

cudaError_t launch_composite_fwd(const BatchParams& bp, const VoxRec* rec, const uint32_t* pair_val,
                                 const uint8_t* pair_mask, const uint2* tile_range, const uint32_t* vis_start,
                                 const uint32_t* tile_order, uint32_t* n_seg, float* t_final,
                                 unsigned long long* work, const Fork* fk, cudaStream_t s) {
    if (bp.n_tiles <= 0) return cudaSuccess;
    if (bp.normals)
        composite_fwd_k<true>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, n_seg, t_final, work,
                              fk, s);
    else
        composite_fwd_k<false>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, n_seg, t_final, work,
                               fk, s);
    return cudaGetLastError();
}

cudaError_t launch_composite_bwd(const BatchParams& bp, const VoxRec* rec, const uint32_t* pair_val,
                                 const uint8_t* pair_mask, const uint2* tile_range, const uint32_t* vis_start,
                                 const uint32_t* tile_order, const float* t_final, const float* g_rgb,
                                 const float* g_depth, const float* g_alpha, const float* g_normal, float* grad_rec,
                                 const Fork* fk, cudaStream_t s) {
    if (bp.n_tiles <= 0) return cudaSuccess;
    if (g_normal)
        composite_bwd_k<true>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, t_final, g_rgb,
                              g_depth, g_alpha, g_normal, grad_rec, fk, s);
    else
        composite_bwd_k<false>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, t_final, g_rgb,
                               g_depth, g_alpha, nullptr, grad_rec, fk, s);
    return cudaGetLastError();
}

cudaError_t launch_composite_export(const BatchParams& bp, const VoxRec* rec, const uint32_t* pair_val,
                                    const uint8_t* pair_mask, const uint2* tile_range, const uint32_t* vis_start,
                                    const uint32_t* tile_order, const int64_t* offsets, uint32_t* voxel, float* weight,
                                    const Fork* fk, cudaStream_t s) {
    if (bp.n_tiles <= 0) return cudaSuccess;
    if (bp.K == 1)
        composite_launch<false, 1, false, true>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, nullptr,
                                                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, offsets,
                                                voxel, weight, fk, s);
    else
        composite_launch<false, 0, false, true>(bp, rec, pair_val, pair_mask, tile_range, vis_start, tile_order, nullptr,
                                                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, offsets,
                                                voxel, weight, fk, s);
    return cudaGetLastError();
}

cudaError_t launch_sh_bwd(const BatchParams& bp, const uint32_t* sorted_g, int64_t n_vis, const VoxRec* rec,
                          const float* grad_rec, bool with_normals, float* const* d_dens, float* const* d_sh,
                          cudaStream_t s) {
    if (n_vis <= 0) return cudaSuccess;
    ShBwdParams sp;
    sp.bp = bp;
    for (int o = 0; o < DV_MAX_OCTREES; ++o) {
        sp.d_dens[o] = (d_dens && o < bp.n_oct) ? d_dens[o] : nullptr;
        sp.d_sh[o] = (d_sh && o < bp.n_oct) ? d_sh[o] : nullptr;
    }
    if (with_normals)
        launch_pdl(k_sh_bwd<true>, dim3((unsigned)((n_vis + 255) / 256)), dim3(256), s, sp, sorted_g, n_vis, rec, grad_rec);
    else
        launch_pdl(k_sh_bwd<false>, dim3((unsigned)((n_vis + 255) / 256)), dim3(256), s, sp, sorted_g, n_vis, rec, grad_rec);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dv
