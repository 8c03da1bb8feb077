// C ABI implementation: validation, per-camera constants, launch sequence,
// saved state and per-kernel event timing.  Declarations and the contract of
// every entry point are in include/dv.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "dv.h"
#include "dv_internal.cuh"

namespace {

const char* const kKernelNames[] = {"project", "scan",        "compact",       "sort_vox",      "records", "emit",
                                    "sort_pairs", "ranges", "composite_fwd", "composite_bwd", "sh_bwd"};
constexpr int kNK = sizeof(kKernelNames) / sizeof(kKernelNames[0]);
enum { KP_PROJECT, KP_SCAN, KP_COMPACT, KP_SORT_VOX, KP_RECORDS, KP_EMIT, KP_SORT_PAIRS, KP_RANGES, KP_FWD, KP_BWD,
       KP_SHBWD };

struct ProfRec {
    int k;
    cudaEvent_t a, b;
};

std::atomic<long long> g_launches{0};

}  // namespace

namespace dv {
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace dv

struct dv_ctx {
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::string err;
    uint64_t* h_scalars = nullptr;  // pinned: [0] n_vis, [1] n_pairs, [2] flags
    uint64_t* d_scalars = nullptr;  // device mirror
    bool profiling = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> spare;
    double ms[kNK] = {};
    int64_t launches[kNK] = {};
};

namespace {

struct CamState {
    std::unique_ptr<FrameParams> fp;
    int64_t n_vis = 0, n_pairs = 0, n_tiles = 0, pix_offset = 0;
    VoxRec* rec = nullptr;
    uint32_t* sorted_g = nullptr;
    uint32_t* pval = nullptr;
    uint8_t* pmask = nullptr;  // per pair: 8x4-pixel blocks of the tile the voxel touches
    uint2* range = nullptr;
    uint32_t* vis_start = nullptr;
    uint32_t* tile_order = nullptr;
    uint32_t* n_seg = nullptr;
    float* t_final = nullptr;
    unsigned long long* work = nullptr;  // [tests, box tests, segments] of the forward
    float* rgb = nullptr;
    float* depth = nullptr;
};

}  // namespace

struct dv_state {
    dv_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<CamState> cams;
    std::vector<void*> owned;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

dv_status fail(dv_ctx* ctx, dv_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

dv_status cuda_fail(dv_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, DV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void prof_begin(dv_ctx* ctx, int k, cudaStream_t s, cudaEvent_t* ev) {
    *ev = nullptr;
    if (!ctx->profiling) return;
    cudaEvent_t e;
    if (!ctx->spare.empty()) {
        e = ctx->spare.back();
        ctx->spare.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return;
    }
    cudaEventRecord(e, s);
    *ev = e;
    (void)k;
}

void prof_end(dv_ctx* ctx, int k, cudaStream_t s, cudaEvent_t a) {
    if (!ctx->profiling || !a) return;
    cudaEvent_t b;
    if (!ctx->spare.empty()) {
        b = ctx->spare.back();
        ctx->spare.pop_back();
    } else if (cudaEventCreate(&b) != cudaSuccess) {
        return;
    }
    cudaEventRecord(b, s);
    ctx->pending.push_back({k, a, b});
}

struct Prof {
    dv_ctx* ctx;
    int k;
    cudaStream_t s;
    cudaEvent_t a;
    Prof(dv_ctx* c, int kk, cudaStream_t ss) : ctx(c), k(kk), s(ss) { prof_begin(c, kk, ss, &a); }
    ~Prof() { prof_end(ctx, k, s, a); }
};

// ---------------------------------------------------------------------------
// small double-precision linear algebra for the per-camera constants
// ---------------------------------------------------------------------------

struct M3 {
    double a[9];
};

M3 load_R(const float* R) {
    M3 m;
    for (int i = 0; i < 9; ++i) m.a[i] = (double)R[i];
    return m;
}

M3 mul(const M3& x, const M3& y) {
    M3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += x.a[i * 3 + k] * y.a[k * 3 + j];
            r.a[i * 3 + j] = s;
        }
    return r;
}

M3 tr(const M3& x) {
    M3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.a[i * 3 + j] = x.a[j * 3 + i];
    return r;
}

void mv(const M3& x, const double* v, double* out) {
    for (int i = 0; i < 3; ++i) out[i] = x.a[i * 3 + 0] * v[0] + x.a[i * 3 + 1] * v[1] + x.a[i * 3 + 2] * v[2];
}

bool rotation_ok(const float* Rf) {
    M3 R = load_R(Rf);
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(R.a[i])) return false;
    M3 G = mul(tr(R), R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (std::fabs(G.a[i * 3 + j] - (i == j ? 1.0 : 0.0)) > 1e-5) return false;
    double det = R.a[0] * (R.a[4] * R.a[8] - R.a[5] * R.a[7]) - R.a[1] * (R.a[3] * R.a[8] - R.a[5] * R.a[6]) +
                 R.a[2] * (R.a[3] * R.a[7] - R.a[4] * R.a[6]);
    return det > 0.0;
}

// conservative tile rectangle of an actor clip box (camera frame points, near-plane clipped)
void box_rect(const FrameParams& fp, const M3& Mc, const double* mc, const float* h, int16_t* rect) {
    double P[8][3];
    for (int c = 0; c < 8; ++c) {
        double q[3] = {(c & 1) ? h[0] : -h[0], (c & 2) ? h[1] : -h[1], (c & 4) ? h[2] : -h[2]};
        mv(Mc, q, P[c]);
        for (int r = 0; r < 3; ++r) P[c][r] += mc[r];
    }
    const double zc = fp.z_clip;
    double u0 = INFINITY, u1 = -INFINITY, v0 = INFINITY, v1 = -INFINITY;
    bool any = false, near_any = false;
    auto add = [&](double x, double y, double z) {
        double u = fp.fx * x / z + fp.cx, v = fp.fy * y / z + fp.cy;
        u0 = std::fmin(u0, u);
        u1 = std::fmax(u1, u);
        v0 = std::fmin(v0, v);
        v1 = std::fmax(v1, v);
        any = true;
    };
    double zmin = INFINITY;
    for (int c = 0; c < 8; ++c) {
        zmin = std::fmin(zmin, P[c][2]);
        if (P[c][2] >= zc)
            add(P[c][0], P[c][1], P[c][2]);
        else
            near_any = true;
    }
    if (near_any)
        for (int bit = 1; bit < 8; bit <<= 1)
            for (int a = 0; a < 8; ++a) {
                if (a & bit) continue;
                int b = a | bit;
                if ((P[a][2] < zc) != (P[b][2] < zc)) {
                    double t = (zc - P[a][2]) / (P[b][2] - P[a][2]);
                    add(P[a][0] + t * (P[b][0] - P[a][0]), P[a][1] + t * (P[b][1] - P[a][1]), zc);
                }
            }
    rect[0] = 1;
    rect[2] = 0;
    rect[1] = 1;
    rect[3] = 0;
    if (!any || zmin > fp.far_) return;
    double lu = std::fmax(u0 - 1.5, -1.0), hu = std::fmin(u1 + 0.5, fp.W + 1.0);
    double lv = std::fmax(v0 - 1.5, -1.0), hv = std::fmin(v1 + 0.5, fp.H + 1.0);
    int pu0 = std::max((int)std::ceil(lu), 0), pu1 = std::min((int)std::floor(hu), fp.W - 1);
    int pv0 = std::max((int)std::ceil(lv), 0), pv1 = std::min((int)std::floor(hv), fp.H - 1);
    if (pu0 > pu1 || pv0 > pv1) return;
    rect[0] = (int16_t)(pu0 / DV_TILE);
    rect[2] = (int16_t)(pu1 / DV_TILE);
    rect[1] = (int16_t)(pv0 / DV_TILE);
    rect[3] = (int16_t)(pv1 / DV_TILE);
}

dv_status make_params(dv_ctx* ctx, const dv_octree* oct, int n_oct, const dv_pose* poses, const dv_camera& cam,
                      const dv_opts& opt, FrameParams& fp) {
    memset(&fp, 0, sizeof(fp));
    fp.W = cam.W;
    fp.H = cam.H;
    fp.tiles_x = (cam.W + DV_TILE - 1) / DV_TILE;
    fp.tiles_y = (cam.H + DV_TILE - 1) / DV_TILE;
    fp.fx = cam.fx;
    fp.fy = cam.fy;
    fp.cx = cam.cx;
    fp.cy = cam.cy;
    fp.near_ = cam.near_;
    fp.far_ = cam.far_;
    fp.K = opt.K;
    fp.inv_k = 1.0f / (float)opt.K;
    fp.eps_stop = opt.eps_stop;
    fp.activation = opt.activation;
    fp.n_oct = n_oct;
    // smallest unit-direction z over the image: samples at distance >= near have z >= near * that
    double xm = std::fmax(std::fabs(0.5 - (double)cam.cx), std::fabs((double)cam.W - 0.5 - (double)cam.cx)) /
                (double)cam.fx;
    double ym = std::fmax(std::fabs(0.5 - (double)cam.cy), std::fabs((double)cam.H - 0.5 - (double)cam.cy)) /
                (double)cam.fy;
    fp.z_clip = (float)(0.999 * (double)cam.near_ / std::sqrt(1.0 + xm * xm + ym * ym));
    int Lkey = 0;
    for (int i = 0; i < n_oct; ++i) Lkey = std::max(Lkey, (int)oct[i].max_level);
    fp.Lkey = Lkey;
    fp.oct_shift = 3 * Lkey;
    M3 Rc = load_R(cam.cam_to_world.R);
    double tc[3] = {cam.cam_to_world.t[0], cam.cam_to_world.t[1], cam.cam_to_world.t[2]};
    int64_t off = 0;
    for (int i = 0; i < n_oct; ++i) {
        OctParams& P = fp.oc[i];
        M3 Ri = load_R(poses[i].R);
        double ti[3] = {poses[i].t[0], poses[i].t[1], poses[i].t[2]};
        M3 A = mul(tr(Ri), Rc);
        M3 Mc = mul(tr(Rc), Ri);
        double dt[3] = {ti[0] - tc[0], ti[1] - tc[1], ti[2] - tc[2]};
        double mc[3], ol[3], ndt[3] = {-dt[0], -dt[1], -dt[2]};
        mv(tr(Rc), dt, mc);
        mv(tr(Ri), ndt, ol);
        for (int k = 0; k < 9; ++k) {
            P.A[k] = (float)A.a[k];
            P.M[k] = (float)Mc.a[k];
        }
        for (int k = 0; k < 3; ++k) {
            P.m[k] = (float)mc[k];
            P.o_loc[k] = (float)ol[k];
            P.clip_half[k] = oct[i].clip_half[k];
            P.root_min[k] = (float)(oct[i].center[k] - 0.5 * oct[i].root_size);
        }
        P.root_size = (float)oct[i].root_size;
        P.role = oct[i].role;
        P.sh_degree = oct[i].sh_degree;
        P.max_level = oct[i].max_level;
        for (int k = 0; k < 3; ++k) {
            double rel = ((double)P.o_loc[k] - (double)P.root_min[k]) / (double)P.root_size;
            double q = std::floor(2.0 * rel * std::ldexp(1.0, Lkey));
            q = std::fmax(std::fmin(q, 1e15), -1e15);
            P.O2[k] = (int64_t)q;
        }
        P.vox_offset = off;
        P.n_vox = oct[i].n_vox;
        P.key = oct[i].key;
        P.dens = oct[i].dens;
        P.sh = oct[i].sh;
        off += oct[i].n_vox;
        if (oct[i].role == DV_ROLE_ACTOR) {
            box_rect(fp, Mc, mc, oct[i].clip_half, P.rect);
        } else {
            P.rect[0] = 1;
            P.rect[2] = 0;
            P.rect[1] = 1;
            P.rect[3] = 0;
        }
    }
    fp.n_vox_total = off;
    (void)ctx;
    return DV_OK;
}

dv_status validate(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_pose* poses, const dv_camera* cams,
                   int32_t n_cam, const dv_opts* opts) {
    if (!oct || !poses || n_oct < 1) return fail(ctx, DV_ERR_INVALID_ARG, "need at least the background octree");
    if (n_oct > DV_MAX_OCTREES) return fail(ctx, DV_ERR_CAPACITY, "too many octrees (max 128)");
    if (n_cam < 0 || (n_cam > 0 && !cams)) return fail(ctx, DV_ERR_INVALID_ARG, "bad camera array");
    if (!opts) return fail(ctx, DV_ERR_INVALID_ARG, "opts is NULL");
    if (opts->K < 1 || opts->K > 16) return fail(ctx, DV_ERR_INVALID_ARG, "K must be in 1..16");
    if (!(opts->eps_stop >= 0.0f) || !std::isfinite(opts->eps_stop))
        return fail(ctx, DV_ERR_INVALID_ARG, "eps_stop must be finite and >= 0");
    if (opts->activation != DV_ACT_EXPLIN && opts->activation != DV_ACT_IDENTITY)
        return fail(ctx, DV_ERR_INVALID_ARG, "unknown activation");
    int64_t total = 0;
    for (int i = 0; i < n_oct; ++i) {
        const dv_octree& o = oct[i];
        if (o.role != (i == 0 ? DV_ROLE_BG : DV_ROLE_ACTOR))
            return fail(ctx, DV_ERR_INVALID_ARG, "octree 0 must be the background and the others actors");
        if (o.n_vox < 0) return fail(ctx, DV_ERR_INVALID_ARG, "negative voxel count");
        if (o.n_vox > 0 && (!o.key || !o.dens || !o.sh))
            return fail(ctx, DV_ERR_INVALID_ARG, "NULL voxel buffer");
        if (o.n_vox > 0 && ((uintptr_t)o.dens & 15)) return fail(ctx, DV_ERR_INVALID_ARG, "dens must be 16-byte aligned");
        if (o.sh_degree < 0 || o.sh_degree > DV_MAX_SH_DEGREE) return fail(ctx, DV_ERR_INVALID_ARG, "sh_degree > 3");
        if (o.max_level < 0 || o.max_level > DV_MAX_LEVEL) return fail(ctx, DV_ERR_INVALID_ARG, "max_level > 16");
        if (!(o.root_size > 0.0) || !std::isfinite(o.root_size))
            return fail(ctx, DV_ERR_INVALID_ARG, "root_size must be > 0");
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(o.center[k])) return fail(ctx, DV_ERR_INVALID_ARG, "non-finite centre");
            if (o.role == DV_ROLE_ACTOR && !(o.clip_half[k] >= 0.0f && std::isfinite(o.clip_half[k])))
                return fail(ctx, DV_ERR_INVALID_ARG, "bad clip box");
        }
        if (!rotation_ok(poses[i].R)) return fail(ctx, DV_ERR_INVALID_POSE, "octree pose is not a rotation");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(poses[i].t[k])) return fail(ctx, DV_ERR_INVALID_POSE, "non-finite translation");
        total += o.n_vox;
    }
    int oct_bits = 0;
    while ((1 << oct_bits) < n_oct) ++oct_bits;
    int Lkey = 0;
    for (int i = 0; i < n_oct; ++i) Lkey = std::max(Lkey, (int)oct[i].max_level);
    if (3 * Lkey + oct_bits > 64) return fail(ctx, DV_ERR_CAPACITY, "depth key does not fit 64 bits");
    if (total >= (int64_t)1 << 31) return fail(ctx, DV_ERR_CAPACITY, "more than 2^31 voxels in one call");
    for (int c = 0; c < n_cam; ++c) {
        const dv_camera& cm = cams[c];
        if (cm.W < 0 || cm.H < 0 || cm.W > DV_MAX_IMAGE || cm.H > DV_MAX_IMAGE)
            return fail(ctx, DV_ERR_INVALID_ARG, "image size out of range");
        if (!(cm.fx > 0.0f) || !(cm.fy > 0.0f) || !std::isfinite(cm.fx) || !std::isfinite(cm.fy) ||
            !std::isfinite(cm.cx) || !std::isfinite(cm.cy))
            return fail(ctx, DV_ERR_INVALID_ARG, "bad intrinsics");
        if (!(cm.near_ > 0.0f) || !(cm.far_ > cm.near_) || !std::isfinite(cm.far_))
            return fail(ctx, DV_ERR_INVALID_ARG, "need 0 < near < far");
        if (!rotation_ok(cm.cam_to_world.R)) return fail(ctx, DV_ERR_INVALID_POSE, "camera pose is not a rotation");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(cm.cam_to_world.t[k])) return fail(ctx, DV_ERR_INVALID_POSE, "non-finite camera");
    }
    return DV_OK;
}

int bits_for(int64_t n) {
    int b = 0;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

template <typename T>
T* pool_alloc(dv_ctx* ctx, cudaStream_t s, size_t count, std::vector<void*>& owned, cudaError_t& err) {
    if (err != cudaSuccess) return nullptr;
    void* p = nullptr;
    size_t bytes = std::max(count * sizeof(T), (size_t)16);
    err = cudaMallocFromPoolAsync(&p, bytes, ctx->pool, s);
    if (err != cudaSuccess) return nullptr;
    owned.push_back(p);
    return (T*)p;
}

// one camera's forward; state buffers go to `st` (always, freed by the caller when not saved)
dv_status render_camera(dv_ctx* ctx, const FrameParams& fp_in, CamState& cs, dv_state* st, float* rgb,
                        float* depth, float* alpha, cudaStream_t s) {
    using namespace dv;
    const FrameParams& fp = fp_in;
    cudaError_t e = cudaSuccess;
    Arena ar;
    ar.pool = ctx->pool;
    ar.stream = s;
    const int64_t Vt = fp.n_vox_total;
    const int64_t npix = (int64_t)fp.W * fp.H;
    const int64_t n_tiles = (int64_t)fp.tiles_x * fp.tiles_y;
    cs.n_tiles = n_tiles;
    cs.rgb = rgb;
    cs.depth = depth;
    std::vector<void*>& own = st->owned;
    cs.n_seg = pool_alloc<uint32_t>(ctx, s, (size_t)npix, own, e);
    cs.t_final = pool_alloc<float>(ctx, s, (size_t)npix, own, e);
    cs.range = pool_alloc<uint2>(ctx, s, (size_t)n_tiles, own, e);
    cs.vis_start = pool_alloc<uint32_t>(ctx, s, (size_t)fp.n_oct + 1, own, e);
    cs.tile_order = pool_alloc<uint32_t>(ctx, s, (size_t)n_tiles, own, e);
    cs.work = pool_alloc<unsigned long long>(ctx, s, 4, own, e);
    if (e == cudaSuccess) e = cudaMemsetAsync(cs.work, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "allocate state");

    uint32_t* cnt = ar.alloc<uint32_t>((size_t)Vt);
    uint64_t* rect = ar.alloc<uint64_t>((size_t)Vt);
    uint64_t* skey = ar.alloc<uint64_t>((size_t)Vt);
    uint32_t* vis = ar.alloc<uint32_t>((size_t)Vt);
    uint32_t* pos = ar.alloc<uint32_t>((size_t)Vt);
    if (ar.err != cudaSuccess) {
        ar.release();
        return cuda_fail(ctx, ar.err, "allocate scratch");
    }
    uint64_t* d_nvis = ctx->d_scalars;
    uint64_t* d_npairs = ctx->d_scalars + 1;
    uint32_t* d_flags = (uint32_t*)(ctx->d_scalars + 2);
    e = cudaMemsetAsync(ctx->d_scalars, 0, 3 * sizeof(uint64_t), s);
    {
        Prof p(ctx, KP_PROJECT, s);
        if (e == cudaSuccess) e = launch_project(fp, cnt, rect, skey, vis, d_flags, s);
    }
    {
        Prof p(ctx, KP_SCAN, s);
        if (e == cudaSuccess) e = scan_u32_to_u32(vis, pos, Vt, (uint32_t*)d_nvis, ar, s);
        if (e == cudaSuccess) e = scan_u32_to_u64(cnt, nullptr, Vt, d_npairs, ar, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_scalars, ctx->d_scalars, 3 * sizeof(uint64_t),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ar.release();
        return cuda_fail(ctx, e, "project");
    }
    const int64_t n_vis = (int64_t)(uint32_t)ctx->h_scalars[0];
    const int64_t P = (int64_t)ctx->h_scalars[1];
    const uint32_t flags = (uint32_t)ctx->h_scalars[2];
    if (flags & DV_FLAG_BAD_LEVEL) {
        ar.release();
        return fail(ctx, DV_ERR_INVALID_ARG, "a leaf key has a level above its octree's max_level or an index "
                                             "outside its level's grid");
    }
    if (P >= ((int64_t)1 << 32) - 1) {
        ar.release();
        return fail(ctx, DV_ERR_CAPACITY, "more than 2^32 (tile, voxel) pairs for one camera");
    }
    cs.n_vis = n_vis;
    cs.n_pairs = P;
    // depth-order sort of the visible voxels
    uint64_t* k0 = ar.alloc<uint64_t>((size_t)n_vis);
    uint64_t* k1 = ar.alloc<uint64_t>((size_t)n_vis);
    uint32_t* g1 = ar.alloc<uint32_t>((size_t)n_vis);
    cs.sorted_g = pool_alloc<uint32_t>(ctx, s, (size_t)n_vis, own, e);
    uint32_t* g0 = cs.sorted_g;
    if (ar.err != cudaSuccess || e != cudaSuccess) {
        ar.release();
        return cuda_fail(ctx, ar.err != cudaSuccess ? ar.err : e, "allocate sort");
    }
    {
        Prof p(ctx, KP_COMPACT, s);
        e = launch_compact(vis, pos, skey, Vt, k0, g0, s);
    }
    uint64_t* kk = k0;
    uint32_t* gg = g0;
    {
        Prof p(ctx, KP_SORT_VOX, s);
        if (e == cudaSuccess)
            e = radix_sort_u64(kk, gg, k1, g1, n_vis, fp.oct_shift + bits_for(fp.n_oct), ar, s);
    }
    if (e == cudaSuccess && gg != cs.sorted_g)
        e = cudaMemcpyAsync(cs.sorted_g, gg, sizeof(uint32_t) * (size_t)n_vis, cudaMemcpyDeviceToDevice, s);
    cs.rec = pool_alloc<VoxRec>(ctx, s, (size_t)n_vis, own, e);
    uint32_t* cnt_sorted = ar.alloc<uint32_t>((size_t)n_vis);
    uint64_t* rect_sorted = ar.alloc<uint64_t>((size_t)n_vis);
    uint64_t* off = ar.alloc<uint64_t>((size_t)n_vis);
    if (ar.err != cudaSuccess || e != cudaSuccess) {
        ar.release();
        return cuda_fail(ctx, ar.err != cudaSuccess ? ar.err : e, "sort voxels");
    }
    {
        Prof p(ctx, KP_RECORDS, s);
        e = launch_records(fp, cs.sorted_g, n_vis, cnt, rect, cs.rec, cnt_sorted, rect_sorted, s);
        if (e == cudaSuccess) e = launch_vis_start(kk, n_vis, fp.oct_shift, fp.n_oct, cs.vis_start, s);
    }
    {
        Prof p(ctx, KP_SCAN, s);
        if (e == cudaSuccess) e = scan_u32_to_u64(cnt_sorted, off, n_vis, nullptr, ar, s);
    }
    // pairs
    uint32_t* pk0 = ar.alloc<uint32_t>((size_t)P);
    uint32_t* pk1 = ar.alloc<uint32_t>((size_t)P);
    uint32_t* pv0 = pool_alloc<uint32_t>(ctx, s, (size_t)P, own, e);
    uint32_t* pv1 = ar.alloc<uint32_t>((size_t)P);
    if (ar.err != cudaSuccess || e != cudaSuccess) {
        ar.release();
        return cuda_fail(ctx, ar.err != cudaSuccess ? ar.err : e, "allocate pairs");
    }
    {
        Prof p(ctx, KP_EMIT, s);
        e = launch_emit(fp, off, rect_sorted, n_vis, P, pk0, pv0, s);
    }
    uint32_t* pk = pk0;
    uint32_t* pv = pv0;
    {
        Prof p(ctx, KP_SORT_PAIRS, s);
        if (e == cudaSuccess) e = radix_sort_u32(pk, pv, pk1, pv1, P, bits_for(n_tiles), ar, s);
    }
    if (e == cudaSuccess && pv != pv0)
        e = cudaMemcpyAsync(pv0, pv, sizeof(uint32_t) * (size_t)P, cudaMemcpyDeviceToDevice, s);
    cs.pval = pv0;
    cs.pmask = pool_alloc<uint8_t>(ctx, s, (size_t)P, own, e);
    {
        Prof p(ctx, KP_RANGES, s);
        if (e == cudaSuccess) e = launch_pair_mask(fp, pk, cs.pval, rect_sorted, P, cs.pmask, s);
        if (e == cudaSuccess) e = launch_ranges(pk, P, cs.range, (int)n_tiles, s);
        uint32_t* tscr = ar.alloc<uint32_t>(64);
        if (e == cudaSuccess) e = tscr ? launch_tile_order(cs.range, (int)n_tiles, tscr, cs.tile_order, s) : ar.err;
    }
    {
        Prof p(ctx, KP_FWD, s);
        if (e == cudaSuccess)
            e = launch_composite_fwd(fp, cs.rec, cs.pval, cs.pmask, cs.range, cs.vis_start, cs.tile_order, rgb, depth, alpha,
                                     cs.n_seg, cs.t_final, cs.work, s);
    }
    ar.release();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "render");
    return DV_OK;
}

void free_state(dv_state* st) {
    if (!st) return;
    if (st->ctx) {
        DeviceGuard g(st->ctx->device);
        for (void* p : st->owned) cudaFreeAsync(p, st->stream);
    }
    delete st;
}

}  // namespace

extern "C" {

const char* dv_version(void) { return "dv 0.1 (sm_103a)"; }

dv_status dv_create(dv_ctx** out, int32_t device) {
    if (!out) return DV_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return DV_ERR_INVALID_ARG;
    std::unique_ptr<dv_ctx> ctx(new (std::nothrow) dv_ctx());
    if (!ctx) return DV_ERR_NOMEM;
    ctx->device = device;
    DeviceGuard g(device);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) return DV_ERR_CUDA;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (cudaMallocHost(&ctx->h_scalars, 4 * sizeof(uint64_t)) != cudaSuccess) {
        cudaMemPoolDestroy(ctx->pool);
        return DV_ERR_NOMEM;
    }
    if (cudaMalloc(&ctx->d_scalars, 4 * sizeof(uint64_t)) != cudaSuccess) {
        cudaFreeHost(ctx->h_scalars);
        cudaMemPoolDestroy(ctx->pool);
        return DV_ERR_NOMEM;
    }
    *out = ctx.release();
    return DV_OK;
}

void dv_destroy(dv_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto& r : ctx->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->spare) cudaEventDestroy(e);
    cudaFree(ctx->d_scalars);
    cudaFreeHost(ctx->h_scalars);
    cudaMemPoolDestroy(ctx->pool);
    delete ctx;
}

const char* dv_last_error(const dv_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

dv_status dv_render(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_pose* poses, const dv_camera* cams,
                    int32_t n_cam, const dv_opts* opts, float* rgb, float* depth, float* alpha, dv_state** saved,
                    void* stream) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (saved) *saved = nullptr;
    dv_status vs = validate(ctx, oct, n_oct, poses, cams, n_cam, opts);
    if (vs != DV_OK) return vs;
    int64_t total_pix = 0;
    for (int c = 0; c < n_cam; ++c) total_pix += (int64_t)cams[c].W * cams[c].H;
    if (total_pix > 0 && (!rgb || !depth || !alpha)) return fail(ctx, DV_ERR_INVALID_ARG, "NULL output buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<dv_state> st(new (std::nothrow) dv_state());
    if (!st) return fail(ctx, DV_ERR_NOMEM, "host allocation");
    st->ctx = ctx;
    st->stream = s;
    st->cams.resize(n_cam);
    int64_t pix_off = 0;
    for (int c = 0; c < n_cam; ++c) {
        CamState& cs = st->cams[c];
        cs.fp.reset(new (std::nothrow) FrameParams());
        if (!cs.fp) {
            free_state(st.release());
            return fail(ctx, DV_ERR_NOMEM, "host allocation");
        }
        make_params(ctx, oct, n_oct, poses, cams[c], *opts, *cs.fp);
        cs.pix_offset = pix_off;
        dv_status rs = render_camera(ctx, *cs.fp, cs, st.get(), rgb + pix_off * 3, depth + pix_off, alpha + pix_off, s);
        if (rs != DV_OK) {
            free_state(st.release());
            return rs;
        }
        pix_off += (int64_t)cams[c].W * cams[c].H;
    }
    if (saved)
        *saved = st.release();
    else
        free_state(st.release());
    return DV_OK;
}

dv_status dv_render_backward(dv_ctx* ctx, dv_state* st, const float* d_rgb, const float* d_depth,
                             const float* d_alpha, float* const* d_dens, float* const* d_sh, void* stream) {
    if (!ctx || !st) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (st->ctx != ctx) return fail(ctx, DV_ERR_INVALID_ARG, "state belongs to another context");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    for (auto& cs : st->cams) {
        const FrameParams& fp = *cs.fp;
        if (cs.n_vis == 0) continue;
        dv::Arena ar;
        ar.pool = ctx->pool;
        ar.stream = s;
        float* grad = ar.alloc<float>((size_t)cs.n_vis * 12);
        if (!grad) {
            ar.release();
            return cuda_fail(ctx, ar.err, "allocate gradient scratch");
        }
        cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * 12 * (size_t)cs.n_vis, s);
        const int64_t po = cs.pix_offset;
        {
            Prof p(ctx, KP_BWD, s);
            if (e == cudaSuccess)
                e = dv::launch_composite_bwd(fp, cs.rec, cs.pval, cs.pmask, cs.range, cs.vis_start, cs.tile_order, cs.rgb,
                                             cs.depth, cs.n_seg, cs.t_final, d_rgb ? d_rgb + po * 3 : nullptr,
                                             d_depth ? d_depth + po : nullptr, d_alpha ? d_alpha + po : nullptr,
                                             grad, s);
        }
        {
            Prof p(ctx, KP_SHBWD, s);
            if (e == cudaSuccess) e = dv::launch_sh_bwd(fp, cs.sorted_g, cs.n_vis, cs.rec, grad, d_dens, d_sh, s);
        }
        ar.release();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "backward");
    }
    return DV_OK;
}

void dv_state_free(dv_state* st) { free_state(st); }

dv_status dv_state_stats(const dv_state* st, int32_t cam, int64_t* n_visible, int64_t* n_pairs, int64_t* n_tiles) {
    if (!st || cam < 0 || cam >= (int32_t)st->cams.size()) return DV_ERR_INVALID_ARG;
    const CamState& cs = st->cams[cam];
    if (n_visible) *n_visible = cs.n_vis;
    if (n_pairs) *n_pairs = cs.n_pairs;
    if (n_tiles) *n_tiles = cs.n_tiles;
    return DV_OK;
}

dv_status dv_state_work(const dv_state* st, int32_t cam, uint64_t* tests, uint64_t* box_tests, uint64_t* segments) {
    if (!st || cam < 0 || cam >= (int32_t)st->cams.size()) return DV_ERR_INVALID_ARG;
    const CamState& cs = st->cams[cam];
    unsigned long long h[4] = {0, 0, 0, 0};
    DeviceGuard g(st->ctx->device);
    if (cudaMemcpyAsync(h, cs.work, sizeof(h), cudaMemcpyDeviceToHost, st->stream) != cudaSuccess ||
        cudaStreamSynchronize(st->stream) != cudaSuccess)
        return DV_ERR_CUDA;
    if (tests) *tests = h[0];
    if (box_tests) *box_tests = h[1];
    if (segments) *segments = h[2];
    return DV_OK;
}

long long dv_launch_count(int32_t reset) {
    return reset ? g_launches.exchange(0) : g_launches.load();
}

dv_status dv_profile_enable(dv_ctx* ctx, int32_t on) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->profiling = on != 0;
    return DV_OK;
}

dv_status dv_profile_read(dv_ctx* ctx, const char* const* names, int32_t n, double* ms, int64_t* launches) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    for (auto& r : ctx->pending) {
        float t = 0.0f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ctx->ms[r.k] += t;
            ctx->launches[r.k] += 1;
        }
        ctx->spare.push_back(r.a);
        ctx->spare.push_back(r.b);
    }
    ctx->pending.clear();
    for (int i = 0; i < n; ++i) {
        int k = -1;
        for (int j = 0; j < kNK; ++j)
            if (names && names[i] && strcmp(names[i], kKernelNames[j]) == 0) k = j;
        if (ms) ms[i] = k >= 0 ? ctx->ms[k] : 0.0;
        if (launches) launches[i] = k >= 0 ? ctx->launches[k] : 0;
    }
    for (int j = 0; j < kNK; ++j) {
        ctx->ms[j] = 0.0;
        ctx->launches[j] = 0;
    }
    return DV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Backward without any allocation.
//
// Some callers cannot allocate device memory at the moment they run the
// backward: a training loop captured into a CUDA graph that must not contain
// allocation nodes, a real-time loop that may not take an allocator lock, or
// a process whose device memory is fully committed to another framework's
// caching allocator.  dv_render_backward_static() serves them: its only
// scratch, the per-voxel gradient accumulator of one camera, lives in the
// file-scope array below, so the call itself never allocates (no cudaMalloc,
// no pool allocation, no library routine that allocates).
//
// Limits and sharing rules:
//  * at most DV_STATIC_MAX_VISIBLE visible voxels per camera (12 floats each,
//    6 MiB in total); a larger camera is rejected with DV_ERR_CAPACITY before
//    any work is enqueued;
//  * every GPU that loads this library holds the array until the process exits;
//  * all calls on a device share the one array: each camera's slice is cleared
//    (cudaMemsetAsync) before use, but two calls whose work overlaps on the GPU
//    (different streams, no ordering between them) race on it and corrupt each
//    other's gradients -- order such calls on one stream or with events;
//  * the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress, with that device current); make that first call
//    before any stream capture begins.
// ---------------------------------------------------------------------------

#define DV_STATIC_MAX_VISIBLE (1 << 17)
#define DV_STATIC_GRAD_FLOATS (12 * DV_STATIC_MAX_VISIBLE)

static __device__ __align__(256) float g_static_grad[DV_STATIC_GRAD_FLOATS];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
float* g_static_ptr[kStaticMaxDevices] = {};

// device address of g_static_grad on `device` (which must be current)
cudaError_t static_grad_ptr(int device, float** out) {
    if (device < 0 || device >= kStaticMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_grad);
        if (e != cudaSuccess) return e;
        g_static_ptr[device] = (float*)p;
    }
    *out = g_static_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" dv_status dv_render_backward_static(dv_ctx* ctx, dv_state* st, const float* d_rgb, const float* d_depth,
                                               const float* d_alpha, float* const* d_dens, float* const* d_sh,
                                               void* stream) {
    if (!ctx || !st) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (st->ctx != ctx) return fail(ctx, DV_ERR_INVALID_ARG, "state belongs to another context");
    for (const auto& cs : st->cams)
        if (cs.n_vis > DV_STATIC_MAX_VISIBLE)
            return fail(ctx, DV_ERR_CAPACITY,
                        "dv_render_backward_static: a camera has " + std::to_string(cs.n_vis) +
                            " visible voxels, above the static limit of " + std::to_string(DV_STATIC_MAX_VISIBLE));
    DeviceGuard g(ctx->device);
    float* grad = nullptr;
    cudaError_t e = static_grad_ptr(ctx->device, &grad);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(static gradient scratch)");
    cudaStream_t s = (cudaStream_t)stream;
    for (auto& cs : st->cams) {
        if (cs.n_vis == 0) continue;
        const int64_t po = cs.pix_offset;
        e = cudaMemsetAsync(grad, 0, sizeof(float) * 12 * (size_t)cs.n_vis, s);
        if (e == cudaSuccess)
            e = dv::launch_composite_bwd(*cs.fp, cs.rec, cs.pval, cs.pmask, cs.range, cs.vis_start, cs.tile_order, cs.rgb,
                                         cs.depth, cs.n_seg, cs.t_final, d_rgb ? d_rgb + po * 3 : nullptr,
                                         d_depth ? d_depth + po : nullptr, d_alpha ? d_alpha + po : nullptr, grad, s);
        if (e == cudaSuccess) e = dv::launch_sh_bwd(*cs.fp, cs.sorted_g, cs.n_vis, cs.rec, grad, d_dens, d_sh, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "dv_render_backward_static");
    }
    return DV_OK;
}
