// C ABI implementation: validation, per-camera constants, launch sequence,
// saved state and per-kernel event timing.  Declarations and the contract of
// every entry point are in include/dv.h.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
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

const char* const kKernelNames[] = {"project", "sort_vox", "records", "sort_pairs", "ranges", "composite_fwd",
                                    "composite_bwd", "sh_bwd"};
constexpr int kNK = sizeof(kKernelNames) / sizeof(kKernelNames[0]);
enum { KP_PROJECT, KP_SORT_VOX, KP_RECORDS, KP_SORT_PAIRS, KP_RANGES, KP_FWD, KP_BWD, KP_SHBWD };

struct ProfRec {
    int k;
    cudaEvent_t a, b;
};

std::atomic<long long> g_launches{0};

}  // namespace

namespace dv {
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace dv

// Mapped (zero-copy) host words, one per live render state: the render's sorts publish their own
// wait flag into it, so a timeout is reported to the call that had it.
struct StatusSlots {
    static constexpr int kBlock = 512;
    std::mutex mu;
    std::vector<uint64_t*> host, dev;  // blocks of kBlock words: host pointers and their device aliases
    std::vector<int> free_list;        // block * kBlock + word
    std::vector<int> deferred;         // given back before their render's last kernel wrote them
    uint64_t* word(int id) { return host[id / kBlock] + id % kBlock; }
    bool take(uint64_t** h, uint64_t** d, int* id) {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = 0; i < deferred.size();) {
            if (*(volatile uint64_t*)word(deferred[i]) != ~0ull) {
                free_list.push_back(deferred[i]);
                deferred[i] = deferred.back();
                deferred.pop_back();
            } else {
                ++i;
            }
        }
        if (free_list.empty()) {
            uint64_t* hb = nullptr;
            uint64_t* db = nullptr;
            if (cudaHostAlloc(&hb, kBlock * sizeof(uint64_t), cudaHostAllocMapped) != cudaSuccess) return false;
            if (cudaHostGetDevicePointer((void**)&db, hb, 0) != cudaSuccess) {
                cudaFreeHost(hb);
                return false;
            }
            const int b = (int)host.size();
            host.push_back(hb);
            dev.push_back(db);
            for (int i = kBlock - 1; i >= 0; --i) free_list.push_back(b * kBlock + i);
        }
        const int s = free_list.back();
        free_list.pop_back();
        *h = host[s / kBlock] + s % kBlock;
        *d = dev[s / kBlock] + s % kBlock;
        *id = s;
        return true;
    }
    // a slot still waiting for its render's write is reused only once that write has landed
    void give(int id) {
        if (id < 0) return;
        std::lock_guard<std::mutex> lk(mu);
        if (*(volatile uint64_t*)word(id) == ~0ull)
            deferred.push_back(id);
        else
            free_list.push_back(id);
    }
    ~StatusSlots() {
        for (uint64_t* h : host) cudaFreeHost(h);
    }
};

// written into a state's status slot before its render is enqueued; the render's last kernel
// overwrites it with the call's sort flag (0 or 1)
constexpr uint64_t kStatusPending = ~0ull;

struct dv_ctx {
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::string err;
    StatusSlots slots;
    dv::Fork fork;          // extra streams and events of the three-launch compositing passes
    int64_t budget = 0;     // bytes one call may take from the pool (0: no limit), set by dv_reserve
    int64_t last_need = 0;  // bytes the last render call needed (or the part known when it failed)
    uint64_t* h_scalars = nullptr;  // pinned, mapped: [0] n_vis, [1] n_pairs, [2] flags, [3] call number
    uint64_t* h_scalars_dev = nullptr;  // the same host words as the device sees them
    uint64_t* d_scalars = nullptr;  // device counters [4] (the projection's), then the depth keys' digit counts [8][256] u32
    uint64_t size_seq = 0;           // render calls so far: the projection writes it into h_scalars[3] last
    char* h_stage = nullptr;         // pinned staging buffer of the per-call view and octree constants
    size_t stage_cap = 0;
    uint32_t* d_spin_err = nullptr;  // the device's wait-error word
    bool profiling = false;
    uint32_t prof_mask = ~0u;  // stages bracketed by events while profiling (bit k: stage k)
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> spare;
    double ms[kNK] = {};
    int64_t launches[kNK] = {};
};

namespace {

// device buffers of one render call (all views), kept for the backward
struct BatchState {
    BatchParams bp{};
    int64_t n_vis = 0, n_pairs = 0, n_pix = 0;
    ViewParams* d_views = nullptr;
    OctParams* d_octs = nullptr;
    std::vector<ViewParams> h_views;
    VoxRec* rec = nullptr;
    float4* nrm = nullptr;  // per record voxel normal (world), when the call renders normals
    uint32_t* sorted_g = nullptr;
    uint32_t* pval = nullptr;
    uint8_t* pmask = nullptr;  // per pair: 8x4-pixel blocks of the tile the voxel touches
    uint2* range = nullptr;
    uint32_t* vis_start = nullptr;
    uint32_t* tile_order = nullptr;
    uint32_t* n_seg = nullptr;
    float* t_final = nullptr;
    unsigned long long* work = nullptr;  // [tests, box tests, segments] of the forward
    uint64_t* d_sort_err = nullptr;      // device word: a sort of this call ran out of its bounded wait
    uint64_t* h_status = nullptr;        // mapped host slot the call publishes d_sort_err into
    uint64_t* h_status_dev = nullptr;
    int status_id = -1;
    bool published = false;  // the kernel that writes the status slot has been enqueued
};

}  // namespace

struct dv_state {
    dv_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    BatchState b;
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
    if (!ctx->profiling || !((ctx->prof_mask >> k) & 1u)) return;
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

// A pipeline stage: an NVTX range named after the stage (seen by profilers; a no-op without one)
// and, while profiling is enabled, a pair of CUDA events on the stage's stream.
struct Prof {
    dv_ctx* ctx;
    int k;
    cudaStream_t s;
    cudaEvent_t a;
    Prof(dv_ctx* c, int kk, cudaStream_t ss) : ctx(c), k(kk), s(ss) {
        nvtxRangePushA(kKernelNames[kk]);
        prof_begin(c, kk, ss, &a);
    }
    ~Prof() {
        prof_end(ctx, k, s, a);
        nvtxRangePop();
    }
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
void box_rect(const ViewParams& fp, const M3& Mc, const double* mc, const float* h, int16_t* rect) {
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

// constants of one view: ViewParams plus one OctParams per octree
void make_view(const dv_octree* oct, int n_oct, const dv_pose* poses, const dv_camera& cam, int Lkey,
               ViewParams& vp, OctParams* P) {
    memset(&vp, 0, sizeof(vp));
    vp.W = cam.W;
    vp.H = cam.H;
    vp.tiles_x = (cam.W + DV_TILE - 1) / DV_TILE;
    vp.tiles_y = (cam.H + DV_TILE - 1) / DV_TILE;
    vp.fx = cam.fx;
    vp.fy = cam.fy;
    vp.cx = cam.cx;
    vp.cy = cam.cy;
    vp.near_ = cam.near_;
    vp.far_ = cam.far_;
    // smallest unit-direction z over the image: samples at distance >= near have z >= near * that
    double xm = std::fmax(std::fabs(0.5 - (double)cam.cx), std::fabs((double)cam.W - 0.5 - (double)cam.cx)) /
                (double)cam.fx;
    double ym = std::fmax(std::fabs(0.5 - (double)cam.cy), std::fabs((double)cam.H - 0.5 - (double)cam.cy)) /
                (double)cam.fy;
    vp.z_clip = (float)(0.999 * (double)cam.near_ / std::sqrt(1.0 + xm * xm + ym * ym));
    M3 Rc = load_R(cam.cam_to_world.R);
    double tc[3] = {cam.cam_to_world.t[0], cam.cam_to_world.t[1], cam.cam_to_world.t[2]};
    int64_t off = 0;
    for (int i = 0; i < n_oct; ++i) {
        OctParams& Q = P[i];
        memset(&Q, 0, sizeof(Q));
        M3 Ri = load_R(poses[i].R);
        double ti[3] = {poses[i].t[0], poses[i].t[1], poses[i].t[2]};
        M3 A = mul(tr(Ri), Rc);
        M3 Mc = mul(tr(Rc), Ri);
        double dt[3] = {ti[0] - tc[0], ti[1] - tc[1], ti[2] - tc[2]};
        double mc[3], ol[3], ndt[3] = {-dt[0], -dt[1], -dt[2]};
        mv(tr(Rc), dt, mc);
        mv(tr(Ri), ndt, ol);
        for (int k = 0; k < 9; ++k) {
            Q.A[k] = (float)A.a[k];
            Q.M[k] = (float)Mc.a[k];
            Q.Rw[k] = (float)Ri.a[k];
        }
        for (int k = 0; k < 3; ++k) {
            Q.m[k] = (float)mc[k];
            Q.o_loc[k] = (float)ol[k];
            Q.clip_half[k] = oct[i].clip_half[k];
            Q.root_min[k] = (float)(oct[i].center[k] - 0.5 * oct[i].root_size);
        }
        Q.root_size = (float)oct[i].root_size;
        Q.role = oct[i].role;
        Q.sh_degree = oct[i].sh_degree;
        Q.max_level = oct[i].max_level;
        for (int k = 0; k < 3; ++k) {
            double rel = ((double)Q.o_loc[k] - (double)Q.root_min[k]) / (double)Q.root_size;
            double q = std::floor(2.0 * rel * std::ldexp(1.0, Lkey));
            q = std::fmax(std::fmin(q, 1e15), -1e15);
            Q.O2[k] = (int64_t)q;
        }
        Q.vox_offset = off;
        Q.n_vox = oct[i].n_vox;
        Q.key = oct[i].key;
        Q.dens = oct[i].dens;
        Q.sh = oct[i].sh;
        off += oct[i].n_vox;
        if (oct[i].role == DV_ROLE_ACTOR) {
            box_rect(vp, Mc, mc, oct[i].clip_half, Q.rect);
        } else {
            Q.rect[0] = 1;
            Q.rect[2] = 0;
            Q.rect[1] = 1;
            Q.rect[3] = 0;
        }
    }
}

int bits_for(int64_t n) {
    int b = 0;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

dv_status validate_octrees(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_opts* opts) {
    if (!oct || n_oct < 1) return fail(ctx, DV_ERR_INVALID_ARG, "need at least the background octree");
    if (n_oct > DV_MAX_OCTREES) return fail(ctx, DV_ERR_CAPACITY, "too many octrees (max 128)");
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
        total += o.n_vox;
    }
    if (total >= (int64_t)1 << 31) return fail(ctx, DV_ERR_CAPACITY, "more than 2^31 voxels in one call");
    return DV_OK;
}

dv_status validate_view(dv_ctx* ctx, const dv_camera& cm, const dv_pose* poses, int n_oct) {
    if (!poses) return fail(ctx, DV_ERR_INVALID_ARG, "NULL pose array");
    for (int i = 0; i < n_oct; ++i) {
        if (!rotation_ok(poses[i].R)) return fail(ctx, DV_ERR_INVALID_POSE, "octree pose is not a rotation");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(poses[i].t[k])) return fail(ctx, DV_ERR_INVALID_POSE, "non-finite translation");
    }
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
    return DV_OK;
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

// ---------------------------------------------------------------------------
// Device memory one render call takes from the context's pool (an upper bound of its peak: the
// saved state plus the scratch released at the end of the call).  Every allocation is counted
// rounded up to 512 bytes.
// ---------------------------------------------------------------------------

int64_t rounded(int64_t bytes) { return ((std::max<int64_t>(bytes, 16) + 511) / 512) * 512; }

// Buffers carved out of one pool allocation, each starting on a 512-byte boundary.  A part
// registered with a null destination only counts toward the size.
struct Layout {
    struct Part {
        void** p;
        int64_t off;
    };
    std::vector<Part> parts;
    int64_t bytes = 0;
    template <typename T>
    void add(T** p, int64_t count) {
        if (p) parts.push_back({reinterpret_cast<void**>(p), bytes});
        bytes += rounded(count * (int64_t)sizeof(T));
    }
    void place(void* base) {
        for (const Part& q : parts) *q.p = static_cast<char*>(base) + q.off;
    }
};

// The four blocks of one render call.  Kept in the saved state: (1) what is known before any work
// is enqueued, (3) what the projection's sizes fix.  Scratch released at the end of the call: (2)
// the projection's per-(view, voxel) arrays and the depth sort's input, (4) the sorts' other
// buffers, the pairs before their sort, and the zero-initialised counters and look-back words.
struct StateBuffers0 {
    ViewParams* views = nullptr;
    OctParams* octs = nullptr;
    uint32_t* n_seg = nullptr;
    float* t_final = nullptr;
    uint2* range = nullptr;
    uint32_t* vis_start = nullptr;
    uint32_t* tile_order = nullptr;
    unsigned long long* work = nullptr;  // [0..3] work counters, [4] the call's sort flag
};

Layout state0_layout(int64_t n_view, int64_t n_oct, int64_t tiles, int64_t pix, StateBuffers0* b) {
    Layout L;
    L.add(b ? &b->views : nullptr, n_view);
    L.add(b ? &b->octs : nullptr, n_view * n_oct);
    L.add(b ? &b->n_seg : nullptr, pix);
    L.add(b ? &b->t_final : nullptr, pix);
    L.add(b ? &b->range : nullptr, tiles);
    L.add(b ? &b->vis_start : nullptr, n_view * n_oct + 1);
    L.add(b ? &b->tile_order : nullptr, tiles);
    L.add(b ? &b->work : nullptr, 5);
    return L;
}

struct PreBuffers {
    uint32_t* cnt = nullptr;   // [NT] tiles of a visible (view, voxel)
    uint64_t* rect = nullptr;  // [NT] its pixel rectangle
    uint64_t* key = nullptr;   // [NT] depth keys of the visible ones, appended
    uint32_t* g = nullptr;     // [NT] their (view, voxel) indices
};

Layout pre_layout(int64_t NT, PreBuffers* b) {
    Layout L;
    L.add(b ? &b->cnt : nullptr, NT);
    L.add(b ? &b->rect : nullptr, NT);
    L.add(b ? &b->key : nullptr, NT);
    L.add(b ? &b->g : nullptr, NT);
    return L;
}

struct StateBuffers1 {
    uint32_t* sorted_g = nullptr;
    VoxRec* rec = nullptr;
    float4* nrm = nullptr;
    uint32_t* pval = nullptr;
    uint8_t* pmask = nullptr;
};

Layout state1_layout(int64_t n_vis, int64_t P, bool normals, StateBuffers1* b) {
    Layout L;
    L.add(b ? &b->sorted_g : nullptr, n_vis);
    L.add(b ? &b->rec : nullptr, n_vis);
    if (normals) L.add(b ? &b->nrm : nullptr, n_vis);
    L.add(b ? &b->pval : nullptr, P);
    L.add(b ? &b->pmask : nullptr, P);
    return L;
}

struct PostBuffers {
    uint64_t* key_tmp = nullptr;      // [n_vis] depth sort ping-pong
    uint32_t* g_tmp = nullptr;        // [n_vis]
    uint64_t* rect_sorted = nullptr;  // [n_vis]
    uint32_t* pk0 = nullptr;          // [P] pair keys (tiles) and their ping-pong
    uint32_t* pk1 = nullptr;
    uint32_t* pv0 = nullptr;          // [P] pair values (records) and their ping-pong
    uint32_t* pv1 = nullptr;
    uint8_t* bucket = nullptr;        // [tiles]
    unsigned long long* zero = nullptr;  // zeroed: look-back words of the records, then the u32 words below
    int64_t zero_bytes = 0;
    // inside `zero`
    unsigned long long* lb_status = nullptr;
    uint32_t* vsort_words = nullptr;
    uint32_t* psort_words = nullptr;
    uint32_t* pair_hist = nullptr;
    uint32_t* ticket = nullptr;
    uint32_t* tile_scratch = nullptr;  // [192] bucket counts and cursors of the tile order
    uint32_t* tile_cnt = nullptr;
};

Layout post_layout(int64_t n_vis, int64_t P, int64_t tiles, int key_bits, int tile_bits, PostBuffers* b) {
    Layout L;
    L.add(b ? &b->key_tmp : nullptr, n_vis);
    L.add(b ? &b->g_tmp : nullptr, n_vis);
    L.add(b ? &b->rect_sorted : nullptr, n_vis);
    L.add(b ? &b->pk0 : nullptr, P);
    L.add(b ? &b->pk1 : nullptr, P);
    L.add(b ? &b->pv0 : nullptr, P);
    L.add(b ? &b->pv1 : nullptr, P);
    L.add(b ? &b->bucket : nullptr, tiles);
    const int64_t n_lb = dv::records_emit_blocks(n_vis);
    const int64_t vw = dv::sort_counted_words(n_vis, key_bits), pw = dv::sort_counted_words(P, tile_bits);
    const int64_t hw = (int64_t)dv::key_passes(tile_bits) * 256;
    const int64_t words32 = vw + pw + hw + 1 + 192 + tiles;
    const int64_t zb = 8 * n_lb + 4 * words32;
    L.add(b ? &b->zero : nullptr, (zb + 7) / 8);
    if (b) b->zero_bytes = zb;
    return L;
}

// pointers inside the zeroed part, once it is placed
void post_place_zero(int64_t n_vis, int64_t P, int key_bits, int tile_bits, PostBuffers& b) {
    b.lb_status = b.zero;
    uint32_t* w = reinterpret_cast<uint32_t*>(b.zero + dv::records_emit_blocks(n_vis));
    b.vsort_words = w;
    w += dv::sort_counted_words(n_vis, key_bits);
    b.psort_words = w;
    w += dv::sort_counted_words(P, tile_bits);
    b.pair_hist = w;
    w += dv::key_passes(tile_bits) * 256;
    b.ticket = w;
    b.tile_scratch = w + 1;
    b.tile_cnt = w + 1 + 192;
}

// the part known before any work is enqueued: per-view constants, per-pixel and per-tile state,
// the projection's per-(view, voxel) arrays
int64_t need_before(int64_t n_view, int64_t n_oct, int64_t NT, int64_t tiles, int64_t pix) {
    return state0_layout(n_view, n_oct, tiles, pix, nullptr).bytes + pre_layout(NT, nullptr).bytes;
}

// the part that follows from the sizes the projection reports: visible voxels and pairs
int64_t need_after(int64_t n_vis, int64_t P, int64_t tiles, int key_bits, int tile_bits, bool normals) {
    return state1_layout(n_vis, P, normals, nullptr).bytes +
           post_layout(n_vis, P, tiles, key_bits, tile_bits, nullptr).bytes;
}

}  // namespace

namespace dv {
int64_t render_need_before(int64_t n_view, int64_t n_oct, int64_t NT, int64_t tiles, int64_t pix) {
    return need_before(n_view, n_oct, NT, tiles, pix);
}
int64_t render_need_after(int64_t n_vis, int64_t P, int64_t tiles, int key_bits, int tile_bits, bool normals) {
    return need_after(n_vis, P, tiles, key_bits, tile_bits, normals);
}
}  // namespace dv

namespace {

// Room for `bytes` in the context's pinned staging buffer (no copy out of it is pending: every call
// that filled it has seen its sizes or waited for its stream).
cudaError_t stage_reserve(dv_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->stage_cap) return cudaSuccess;
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->stage_cap = 0;
    const size_t cap = std::max<size_t>(bytes, 64 << 10);
    const cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&ctx->h_stage), cap, cudaHostAllocDefault);
    if (e == cudaSuccess) ctx->stage_cap = cap;
    return e;
}

// Waits until the projection has written this call's sizes: its last block stores the call number
// into h_scalars[3] after the sizes, so polling that word ends as soon as they are there; querying
// the stream now and then reports a kernel that failed.
cudaError_t wait_sizes(dv_ctx* ctx, uint64_t seq, cudaStream_t s) {
    for (uint32_t i = 1;; ++i) {
        if (__atomic_load_n(ctx->h_scalars + 3, __ATOMIC_ACQUIRE) == seq) return cudaSuccess;
        if ((i & 255u) == 0) {
            const cudaError_t q = cudaStreamQuery(s);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return q;
            return __atomic_load_n(ctx->h_scalars + 3, __ATOMIC_ACQUIRE) == seq ? cudaSuccess : cudaErrorUnknown;
        }
    }
}

// The forward of one render call over all its views.  State buffers go to `st`
// (freed by the caller when no state is wanted).
dv_status render_batch(dv_ctx* ctx, const dv_octree* oct, int n_oct, const dv_pose* const* view_poses,
                       const dv_camera* cams, int n_view, const dv_opts& opt, dv_state* st, float* const* rgbs,
                       float* const* depths, float* const* alphas, float* const* normals, cudaStream_t s) {
    using namespace dv;
    BatchState& B = st->b;
    BatchParams& bp = B.bp;
    memset(&bp, 0, sizeof(bp));
    bp.n_view = n_view;
    bp.n_oct = n_oct;
    bp.K = opt.K;
    bp.inv_k = 1.0f / (float)opt.K;
    bp.eps_stop = opt.eps_stop;
    bp.normals = normals ? 1 : 0;
    bp.activation = opt.activation;
    int Lkey = 0;
    for (int i = 0; i < n_oct; ++i) Lkey = std::max(Lkey, (int)oct[i].max_level);
    bp.Lkey = Lkey;
    bp.oct_shift = 3 * Lkey;
    bp.view_shift = bp.oct_shift + bits_for(n_oct);
    int64_t off = 0;
    for (int i = 0; i < n_oct; ++i) {
        bp.vox_offset[i] = off;
        off += oct[i].n_vox;
    }
    for (int i = n_oct; i <= DV_MAX_OCTREES; ++i) bp.vox_offset[i] = off;
    bp.n_vox = off;
    // per-view constants
    std::vector<OctParams> h_octs((size_t)n_view * n_oct);
    B.h_views.resize(n_view);
    int64_t tiles = 0, pix = 0;
    for (int v = 0; v < n_view; ++v) {
        make_view(oct, n_oct, view_poses[v], cams[v], Lkey, B.h_views[v], &h_octs[(size_t)v * n_oct]);
        B.h_views[v].tile_base = (int32_t)tiles;
        B.h_views[v].pix_base = pix;
        B.h_views[v].rgb = rgbs[v];
        B.h_views[v].normal = normals ? normals[v] : nullptr;
        B.h_views[v].depth = depths[v];
        B.h_views[v].alpha = alphas[v];
        bp.tile_base[v] = (int32_t)tiles;
        tiles += (int64_t)B.h_views[v].tiles_x * B.h_views[v].tiles_y;
        pix += (int64_t)cams[v].W * cams[v].H;
    }
    for (int v = n_view; v <= DV_MAX_VIEWS; ++v) bp.tile_base[v] = (int32_t)tiles;
    if (tiles >= ((int64_t)1 << 31)) return fail(ctx, DV_ERR_CAPACITY, "too many tiles in one call");
    bp.n_tiles = (int32_t)tiles;
    // tiles by the number of actor clip boxes that cover them (none, 1 to 4, 5 or more): the three
    // groups of the compositing launches; the tile-order kernel classifies each tile by the same rectangles
    {
        int64_t n_large = 0, n_small = 0;
        std::vector<uint8_t> cov;
        for (int v = 0; v < n_view; ++v) {
            const ViewParams& vp = B.h_views[v];
            cov.assign((size_t)vp.tiles_x * vp.tiles_y, 0);
            for (int o = 1; o < n_oct; ++o) {
                const OctParams& Q = h_octs[(size_t)v * n_oct + o];
                if (Q.role != DV_ROLE_ACTOR) continue;
                for (int ty = std::max<int>(Q.rect[1], 0); ty <= std::min<int>(Q.rect[3], vp.tiles_y - 1); ++ty)
                    for (int tx = std::max<int>(Q.rect[0], 0); tx <= std::min<int>(Q.rect[2], vp.tiles_x - 1); ++tx) {
                        uint8_t& c = cov[(size_t)ty * vp.tiles_x + tx];
                        if (c < 5) ++c;
                    }
            }
            for (uint8_t c : cov) {
                n_large += c >= 5;
                n_small += c > 0 && c < 5;
            }
        }
        bp.n_tiles_large = (int32_t)n_large;
        bp.n_tiles_small = (int32_t)n_small;
    }
    B.n_pix = pix;
    const int64_t NT = bp.n_vox * n_view;
    if (NT >= ((int64_t)1 << 32)) return fail(ctx, DV_ERR_CAPACITY, "views x voxels exceeds 2^32");
    const int key_bits = bp.view_shift + bits_for(n_view);
    const int tile_bits = bits_for(tiles);
    const int64_t need0 = need_before(n_view, n_oct, NT, tiles, pix);
    ctx->last_need = need0;
    if (ctx->budget > 0 && need0 > ctx->budget)
        return fail(ctx, DV_ERR_CAPACITY, "the call needs at least " + std::to_string(need0) +
                                              " bytes of workspace, above the reserved " +
                                              std::to_string(ctx->budget) + " (dv_reserve)");
    cudaError_t e = cudaSuccess;
    std::vector<void*>& own = st->owned;
    StateBuffers0 sb0;
    {
        Layout L = state0_layout(n_view, n_oct, tiles, pix, &sb0);
        char* blk = pool_alloc<char>(ctx, s, (size_t)L.bytes, own, e);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "allocate state");
        L.place(blk);
    }
    B.d_views = sb0.views;
    B.d_octs = sb0.octs;
    B.n_seg = sb0.n_seg;
    B.t_final = sb0.t_final;
    B.range = sb0.range;
    B.vis_start = sb0.vis_start;
    B.tile_order = sb0.tile_order;
    B.work = sb0.work;
    B.d_sort_err = reinterpret_cast<uint64_t*>(sb0.work + 4);
    bp.views = B.d_views;
    bp.octs = B.d_octs;
    if (!ctx->slots.take(&B.h_status, &B.h_status_dev, &B.status_id))
        return fail(ctx, DV_ERR_NOMEM, "mapped host memory for the call's status word");
    *(volatile uint64_t*)B.h_status = kStatusPending;
    uint32_t* sort_err = reinterpret_cast<uint32_t*>(B.d_sort_err);

    Arena ar;
    ar.pool = ctx->pool;
    ar.stream = s;
    PreBuffers pre;
    {
        Layout L = pre_layout(NT, &pre);
        char* blk = ar.alloc<char>((size_t)L.bytes);
        if (ar.err != cudaSuccess) {
            ar.release();
            return cuda_fail(ctx, ar.err, "allocate scratch");
        }
        L.place(blk);
    }
    // The view and octree constants in one asynchronous copy from the pinned staging buffer (the
    // two parts sit at the same offsets there as in the state block).  The buffer is free again once
    // this call has seen its sizes (the projection follows the copy on the stream); a call that
    // fails before that waits for its stream, so the next call never overwrites a pending copy.
    const size_t octs_off = (size_t)(reinterpret_cast<char*>(B.d_octs) - reinterpret_cast<char*>(B.d_views));
    const size_t stage_bytes = octs_off + sizeof(OctParams) * h_octs.size();
    e = stage_reserve(ctx, stage_bytes);
    if (e != cudaSuccess) {
        ar.release();
        return cuda_fail(ctx, e, "staging buffer");
    }
    memcpy(ctx->h_stage, B.h_views.data(), sizeof(ViewParams) * n_view);
    memcpy(ctx->h_stage + octs_off, h_octs.data(), sizeof(OctParams) * h_octs.size());
    e = cudaMemcpyAsync(B.d_views, ctx->h_stage, stage_bytes, cudaMemcpyHostToDevice, s);
    // the projection's counters, then the digit counts of the depth keys
    uint32_t* key_hist = reinterpret_cast<uint32_t*>(ctx->d_scalars + 4);
    const uint64_t seq = ++ctx->size_seq;
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->d_scalars, 0, 4 * sizeof(uint64_t) + (size_t)key_passes(key_bits) * 256 * 4, s);
    {
        Prof p(ctx, KP_PROJECT, s);
        if (e == cudaSuccess)
            e = launch_project(bp, pre.cnt, pre.rect, pre.key, pre.g, key_hist, key_bits,
                               (unsigned long long*)ctx->d_scalars, ctx->h_scalars_dev, seq, ctx->d_spin_err,
                               B.work, s);
    }
    // the projection's last block writes the sizes into mapped host memory: no copy engine is
    // involved, so a large device-to-host transfer queued by the caller on another stream cannot
    // delay this read-back
    if (e == cudaSuccess) e = wait_sizes(ctx, seq, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        ar.release();
        return cuda_fail(ctx, e, "project");
    }
    const int64_t n_vis = (int64_t)(uint32_t)ctx->h_scalars[0];
    const int64_t P = (int64_t)ctx->h_scalars[1];
    const uint32_t flags = (uint32_t)ctx->h_scalars[2];
    if (flags & DV_FLAG_SPIN_TIMEOUT) {
        ar.release();
        return fail(ctx, DV_ERR_TIMEOUT, "a radix-sort pass on this device ran out of its bounded look-back wait in an "
                                         "earlier call; that call's results are invalid");
    }
    if (flags & DV_FLAG_BAD_LEVEL) {
        ar.release();
        return fail(ctx, DV_ERR_INVALID_ARG, "a leaf key has a level above its octree's max_level or an index "
                                             "outside its level's grid");
    }
    if (P >= ((int64_t)1 << 32) - 1) {
        ar.release();
        return fail(ctx, DV_ERR_CAPACITY, "more than 2^32 (tile, voxel) pairs in one call");
    }
    {
        const int64_t need = need0 + need_after(n_vis, P, tiles, key_bits, tile_bits, bp.normals != 0);
        ctx->last_need = need;
        if (ctx->budget > 0 && need > ctx->budget) {
            ar.release();
            return fail(ctx, DV_ERR_CAPACITY, "the call needs " + std::to_string(need) +
                                                  " bytes of workspace (" + std::to_string(n_vis) +
                                                  " visible voxels, " + std::to_string(P) +
                                                  " pairs), above the reserved " + std::to_string(ctx->budget) +
                                                  " (dv_reserve); no output was written");
        }
    }
    B.n_vis = n_vis;
    B.n_pairs = P;
    bp.n_vis = n_vis;
    bp.n_pairs = P;
    StateBuffers1 sb1;
    {
        Layout L = state1_layout(n_vis, P, bp.normals != 0, &sb1);
        char* blk = pool_alloc<char>(ctx, s, (size_t)L.bytes, own, e);
        if (e == cudaSuccess) L.place(blk);
    }
    PostBuffers post;
    {
        Layout L = post_layout(n_vis, P, tiles, key_bits, tile_bits, &post);
        char* blk = ar.alloc<char>((size_t)L.bytes);
        if (ar.err == cudaSuccess) {
            L.place(blk);
            post_place_zero(n_vis, P, key_bits, tile_bits, post);
        }
    }
    if (ar.err != cudaSuccess || e != cudaSuccess) {
        ar.release();
        return cuda_fail(ctx, ar.err != cudaSuccess ? ar.err : e, "allocate sort");
    }
    B.sorted_g = sb1.sorted_g;
    B.rec = sb1.rec;
    B.nrm = sb1.nrm;
    B.pval = sb1.pval;
    B.pmask = sb1.pmask;
    bp.sorted_g = B.sorted_g;
    bp.nrm = B.nrm;
    e = cudaMemsetAsync(post.zero, 0, (size_t)post.zero_bytes, s);
    // depth-order sort of the visible (view, voxel)s: the values land in sorted_g
    uint64_t* sorted_key = nullptr;
    {
        Prof p(ctx, KP_SORT_VOX, s);
        if (e == cudaSuccess)
            e = sort_counted_u64(pre.key, pre.g, post.key_tmp, post.g_tmp, sorted_key, B.sorted_g, n_vis, key_bits,
                                 key_hist, post.vsort_words, sort_err, ar, s);
    }
    // records, then the (tile, record) pairs in depth order with their tile counts and digits
    {
        Prof p(ctx, KP_RECORDS, s);
        if (e == cudaSuccess)
            e = launch_records_emit(bp, B.sorted_g, sorted_key, n_vis, P, pre.cnt, pre.rect, B.rec, B.nrm,
                                    post.rect_sorted, B.vis_start, post.pk0, post.pv0, post.pair_hist, tile_bits,
                                    post.tile_cnt, post.lb_status, post.ticket, sort_err, ctx->d_spin_err, s);
    }
    // stable sort of the pairs by tile: every tile's list stays front to back; the values land in pval
    uint32_t* sorted_tile = nullptr;
    {
        Prof p(ctx, KP_SORT_PAIRS, s);
        if (e == cudaSuccess)
            e = sort_counted_u32(post.pk0, post.pv0, post.pk1, post.pv1, sorted_tile, B.pval, P, tile_bits,
                                 post.pair_hist, post.psort_words, sort_err, ar, s);
    }
    {
        Prof p(ctx, KP_RANGES, s);
        // the call's own sort flag goes to its status slot (read by dv_state_check, the backward and
        // the serving loop), so a timeout is reported to the call that had it
        if (e == cudaSuccess)
            e = launch_pair_mask(bp, sorted_tile, B.pval, post.rect_sorted, P, n_vis, B.pmask, B.range,
                                 B.d_sort_err, B.h_status_dev, s);
        if (e == cudaSuccess) B.published = true;
        if (e == cudaSuccess)
            e = launch_tile_order(bp, post.tile_cnt, (int)tiles, B.range, post.bucket, post.tile_scratch,
                                  B.tile_order, s);
    }
    {
        Prof p(ctx, KP_FWD, s);
        if (e == cudaSuccess)
            e = launch_composite_fwd(bp, B.rec, B.pval, B.pmask, B.range, B.vis_start, B.tile_order, B.n_seg,
                                     B.t_final, B.work, &ctx->fork, s);
    }
    ar.release();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "render");
    return DV_OK;
}

// floats per visible voxel of the backward's gradient scratch
size_t grad_stride(bool with_normals) { return with_normals ? 16 : 12; }

// d_normal: dL/dN of a call that rendered normals, or null (no gradient through N)
dv_status backward_batch(dv_ctx* ctx, dv_state* st, const float* d_rgb, const float* d_depth, const float* d_alpha,
                         const float* d_normal, float* const* d_dens, float* const* d_sh, float* grad, cudaStream_t s) {
    BatchState& B = st->b;
    const bool nrm = d_normal != nullptr;
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * grad_stride(nrm) * (size_t)B.n_vis, s);
    {
        Prof p(ctx, KP_BWD, s);
        if (e == cudaSuccess)
            e = dv::launch_composite_bwd(B.bp, B.rec, B.pval, B.pmask, B.range, B.vis_start, B.tile_order, B.t_final,
                                         d_rgb, d_depth, d_alpha, d_normal, grad, &ctx->fork, s);
    }
    {
        Prof p(ctx, KP_SHBWD, s);
        if (e == cudaSuccess) e = dv::launch_sh_bwd(B.bp, B.sorted_g, B.n_vis, B.rec, grad, nrm, d_dens, d_sh, s);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "backward");
    return DV_OK;
}

void free_state(dv_state* st) {
    if (!st) return;
    if (st->ctx) {
        DeviceGuard g(st->ctx->device);
        for (void* p : st->owned) cudaFreeAsync(p, st->stream);
        if (st->b.status_id >= 0 && !st->b.published) *(volatile uint64_t*)st->b.h_status = 0;  // nothing will write it
        st->ctx->slots.give(st->b.status_id);
    }
    delete st;
}

// The call's sort flag as published into its status slot: 1 timed out, 0 fine, kStatusPending
// not yet known (the render has not finished).
uint64_t state_sort_flag(const dv_state* st) {
    if (!st || st->b.status_id < 0) return 0;
    return *(volatile const uint64_t*)st->b.h_status;
}

}  // namespace

extern "C" {

const char* dv_version(void) { return "dv 0.1 (sm_103a)"; }

// The extra streams of the three-launch compositing passes get the device's highest priority: their
// launches hold the tiles that actor boxes cover, the heaviest of a frame, so their CTAs are
// dispatched ahead of the plain launch's and start at once instead of forming a tail behind them.
static int side_priority() {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
    return greatest;
}

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
    if (cudaHostAlloc(&ctx->h_scalars, 4 * sizeof(uint64_t), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&ctx->h_scalars_dev, ctx->h_scalars, 0) != cudaSuccess) {
        if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
        cudaMemPoolDestroy(ctx->pool);
        return DV_ERR_NOMEM;
    }
    memset(ctx->h_scalars, 0, 4 * sizeof(uint64_t));
    if (cudaMalloc(&ctx->d_scalars, 4 * sizeof(uint64_t) + 8 * 256 * sizeof(uint32_t)) != cudaSuccess) {
        cudaFreeHost(ctx->h_scalars);
        cudaMemPoolDestroy(ctx->pool);
        return DV_ERR_NOMEM;
    }
    ctx->d_spin_err = dv::spin_error_word();
    if (!ctx->d_spin_err ||
        cudaStreamCreateWithPriority(&ctx->fork.side, cudaStreamNonBlocking, side_priority()) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ctx->fork.side2, cudaStreamNonBlocking, side_priority()) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork.ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork.ev_join2, cudaEventDisableTiming) != cudaSuccess) {
        if (ctx->fork.ev_fork) cudaEventDestroy(ctx->fork.ev_fork);
        if (ctx->fork.ev_join) cudaEventDestroy(ctx->fork.ev_join);
        if (ctx->fork.side) cudaStreamDestroy(ctx->fork.side);
        if (ctx->fork.side2) cudaStreamDestroy(ctx->fork.side2);
        cudaFree(ctx->d_scalars);
        cudaFreeHost(ctx->h_scalars);
        cudaMemPoolDestroy(ctx->pool);
        return DV_ERR_CUDA;
    }
    *out = ctx.release();
    return DV_OK;
}

dv_status dv_debug_flag_spin_timeout(dv_ctx* ctx) {
    if (!ctx || !ctx->d_spin_err) return DV_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const uint32_t one = 1u;
    const cudaError_t e = cudaMemcpy(ctx->d_spin_err, &one, sizeof(one), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? DV_OK : cuda_fail(ctx, e, "flag spin timeout");
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
    if (ctx->fork.ev_fork) cudaEventDestroy(ctx->fork.ev_fork);
    if (ctx->fork.ev_join) cudaEventDestroy(ctx->fork.ev_join);
    if (ctx->fork.ev_join2) cudaEventDestroy(ctx->fork.ev_join2);
    if (ctx->fork.side) cudaStreamDestroy(ctx->fork.side);
    if (ctx->fork.side2) cudaStreamDestroy(ctx->fork.side2);
    cudaFree(ctx->d_scalars);
    cudaFreeHost(ctx->h_scalars);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    cudaMemPoolDestroy(ctx->pool);
    delete ctx;
}

const char* dv_last_error(const dv_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

static dv_status render_common(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_pose* const* view_poses,
                               const dv_camera* cams, int32_t n_view, const dv_opts* opts, float* rgb, float* depth,
                               float* alpha, float* const* rgbs, float* const* depths, float* const* alphas,
                               dv_state** saved, void* stream, float* normal = nullptr) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (saved) *saved = nullptr;
    dv_status vs = validate_octrees(ctx, oct, n_oct, opts);
    if (vs != DV_OK) return vs;
    if (n_view < 0 || (n_view > 0 && (!cams || !view_poses))) return fail(ctx, DV_ERR_INVALID_ARG, "bad view array");
    if (n_view > DV_MAX_VIEWS) return fail(ctx, DV_ERR_CAPACITY, "too many views in one call (max 64)");
    int64_t total_pix = 0;
    for (int v = 0; v < n_view; ++v) {
        vs = validate_view(ctx, cams[v], view_poses[v], n_oct);
        if (vs != DV_OK) return vs;
        total_pix += (int64_t)cams[v].W * cams[v].H;
    }
    int Lkey = 0;
    for (int i = 0; i < n_oct; ++i) Lkey = std::max(Lkey, (int)oct[i].max_level);
    if (3 * Lkey + bits_for(n_oct) + bits_for(n_view) > 64)
        return fail(ctx, DV_ERR_CAPACITY, "depth key does not fit 64 bits");
    // per-view output pointers: given, or carved from the concatenated buffers
    std::vector<float*> vr((size_t)std::max(n_view, 1)), vd(vr.size()), va(vr.size()), vn(vr.size());
    int64_t pb = 0;
    for (int v = 0; v < n_view; ++v) {
        const int64_t n = (int64_t)cams[v].W * cams[v].H;
        if (rgbs) {
            vr[v] = rgbs[v];
            vd[v] = depths ? depths[v] : nullptr;
            va[v] = alphas ? alphas[v] : nullptr;
        } else {
            vr[v] = rgb ? rgb + pb * 3 : nullptr;
            vd[v] = depth ? depth + pb : nullptr;
            va[v] = alpha ? alpha + pb : nullptr;
        }
        vn[v] = normal ? normal + pb * 3 : nullptr;
        if (n > 0 && (!vr[v] || !vd[v] || !va[v])) return fail(ctx, DV_ERR_INVALID_ARG, "NULL output buffer");
        pb += n;
    }
    (void)total_pix;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<dv_state> st(new (std::nothrow) dv_state());
    if (!st) return fail(ctx, DV_ERR_NOMEM, "host allocation");
    st->ctx = ctx;
    st->stream = s;
    if (n_view > 0) {
        dv_status rs = render_batch(ctx, oct, n_oct, view_poses, cams, n_view, *opts, st.get(), vr.data(), vd.data(),
                                    va.data(), normal ? vn.data() : nullptr, s);
        if (rs != DV_OK) {
            free_state(st.release());
            return rs;
        }
    }
    if (saved)
        *saved = st.release();
    else
        free_state(st.release());
    return DV_OK;
}

dv_status dv_render(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_pose* poses, const dv_camera* cams,
                    int32_t n_cam, const dv_opts* opts, float* rgb, float* depth, float* alpha, dv_state** saved,
                    void* stream) {
    if (n_cam < 0 || n_cam > DV_MAX_VIEWS) {
        if (ctx) ctx->err = "camera count out of range (0..64)";
        return n_cam < 0 ? DV_ERR_INVALID_ARG : DV_ERR_CAPACITY;
    }
    std::vector<const dv_pose*> vp((size_t)std::max(n_cam, 1), poses);
    return render_common(ctx, oct, n_oct, vp.data(), cams, n_cam, opts, rgb, depth, alpha, nullptr, nullptr, nullptr,
                         saved, stream);
}

dv_status dv_render_views(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_view* views, int32_t n_view,
                          const dv_opts* opts, float* rgb, float* depth, float* alpha, dv_state** saved,
                          void* stream) {
    if (n_view < 0 || n_view > DV_MAX_VIEWS || (n_view > 0 && !views)) {
        if (ctx) ctx->err = "view count out of range (0..64) or NULL views";
        return n_view > DV_MAX_VIEWS ? DV_ERR_CAPACITY : DV_ERR_INVALID_ARG;
    }
    std::vector<const dv_pose*> vp((size_t)std::max(n_view, 1), nullptr);
    std::vector<dv_camera> cams((size_t)std::max(n_view, 1));
    for (int v = 0; v < n_view; ++v) {
        vp[v] = views[v].poses;
        cams[v] = views[v].camera;
    }
    return render_common(ctx, oct, n_oct, vp.data(), cams.data(), n_view, opts, rgb, depth, alpha, nullptr, nullptr,
                         nullptr, saved, stream);
}

static dv_status backward_common(dv_ctx* ctx, dv_state* st, const float* d_rgb, const float* d_depth,
                                 const float* d_alpha, const float* d_normal, float* const* d_dens, float* const* d_sh,
                                 void* stream) {
    if (!ctx || !st) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (st->ctx != ctx) return fail(ctx, DV_ERR_INVALID_ARG, "state belongs to another context");
    if (d_normal && !st->b.bp.normals)
        return fail(ctx, DV_ERR_INVALID_ARG, "a normal gradient for a render without normals");
    if (state_sort_flag(st) == 1)
        return fail(ctx, DV_ERR_TIMEOUT, "the render of this state had a sort whose bounded wait ran out; its "
                                         "results are invalid");
    if (st->b.n_vis == 0) return DV_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    dv::Arena ar;
    ar.pool = ctx->pool;
    ar.stream = s;
    float* grad = ar.alloc<float>((size_t)st->b.n_vis * grad_stride(d_normal != nullptr));
    if (!grad) {
        ar.release();
        return cuda_fail(ctx, ar.err, "allocate gradient scratch");
    }
    dv_status r = backward_batch(ctx, st, d_rgb, d_depth, d_alpha, d_normal, d_dens, d_sh, grad, s);
    ar.release();
    return r;
}

dv_status dv_render_backward(dv_ctx* ctx, dv_state* st, const float* d_rgb, const float* d_depth,
                             const float* d_alpha, float* const* d_dens, float* const* d_sh, void* stream) {
    return backward_common(ctx, st, d_rgb, d_depth, d_alpha, nullptr, d_dens, d_sh, stream);
}

dv_status dv_render_normals(dv_ctx* ctx, const dv_octree* oct, int32_t n_oct, const dv_pose* poses,
                            const dv_camera* cams, int32_t n_cam, const dv_opts* opts, float* rgb, float* depth,
                            float* alpha, float* normal, dv_state** saved, void* stream) {
    if (n_cam < 0 || n_cam > DV_MAX_VIEWS) {
        if (ctx) ctx->err = "camera count out of range (0..64)";
        return n_cam < 0 ? DV_ERR_INVALID_ARG : DV_ERR_CAPACITY;
    }
    int64_t pix = 0;
    for (int v = 0; v < n_cam && cams; ++v) pix += (int64_t)cams[v].W * cams[v].H;
    if (pix > 0 && !normal) {
        if (ctx) ctx->err = "NULL normal buffer";
        return DV_ERR_INVALID_ARG;
    }
    std::vector<const dv_pose*> vp((size_t)std::max(n_cam, 1), poses);
    return render_common(ctx, oct, n_oct, vp.data(), cams, n_cam, opts, rgb, depth, alpha, nullptr, nullptr, nullptr,
                         saved, stream, normal);
}

dv_status dv_render_backward_normals(dv_ctx* ctx, dv_state* st, const float* d_rgb, const float* d_depth,
                                     const float* d_alpha, const float* d_normal, float* const* d_dens,
                                     float* const* d_sh, void* stream) {
    return backward_common(ctx, st, d_rgb, d_depth, d_alpha, d_normal, d_dens, d_sh, stream);
}

void dv_state_free(dv_state* st) { free_state(st); }

// ---- compositing weights and feature fields ----

dv_status dv_state_weight_offsets(dv_ctx* ctx, dv_state* st, int64_t* offsets, int64_t* total, void* stream) {
    if (!ctx || !st || !total) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (st->ctx != ctx) return fail(ctx, DV_ERR_INVALID_ARG, "state belongs to another context");
    *total = 0;
    BatchState& B = st->b;
    if (B.n_pix > 0 && !offsets) return fail(ctx, DV_ERR_INVALID_ARG, "NULL offsets");
    if (B.n_pix == 0) return DV_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    dv::Arena ar;
    ar.pool = ctx->pool;
    ar.stream = s;
    cudaError_t e = dv::scan_u32_to_u64(B.n_seg, (uint64_t*)offsets, B.n_pix, (uint64_t*)(offsets + B.n_pix), ar, s);
    ar.release();
    if (e == cudaSuccess) e = cudaMemcpyAsync(total, offsets + B.n_pix, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weight offsets");
    return DV_OK;
}

dv_status dv_state_weights(dv_ctx* ctx, dv_state* st, const int64_t* offsets, uint32_t* voxel, float* weight,
                           void* stream) {
    if (!ctx || !st) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (st->ctx != ctx) return fail(ctx, DV_ERR_INVALID_ARG, "state belongs to another context");
    BatchState& B = st->b;
    if (B.n_pix == 0 || B.n_vis == 0) return DV_OK;
    if (!offsets || !voxel || !weight) return fail(ctx, DV_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaError_t e = dv::launch_composite_export(B.bp, B.rec, B.pval, B.pmask, B.range, B.vis_start, B.tile_order,
                                                offsets, voxel, weight, &ctx->fork, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weights export");
    return DV_OK;
}

dv_status dv_features_render(dv_ctx* ctx, int64_t n_pix, const int64_t* offsets, const uint32_t* voxel,
                             const float* weight, const float* feat, int32_t C, float* out, void* stream) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n_pix < 0 || C < 1 || C > 65536) return fail(ctx, DV_ERR_INVALID_ARG, "bad pixel or channel count");
    if (n_pix > 0 && (!offsets || !feat || !out)) return fail(ctx, DV_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaError_t e = dv::launch_feat_render(n_pix, offsets, voxel, weight, feat, C, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "feature render");
    return DV_OK;
}

dv_status dv_features_fuse(dv_ctx* ctx, int64_t n_pix, const int64_t* offsets, const uint32_t* voxel,
                           const float* weight, const float* feat2d, int32_t C, float* accum, float* wsum,
                           void* stream) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n_pix < 0 || C < 1 || C > 65536) return fail(ctx, DV_ERR_INVALID_ARG, "bad pixel or channel count");
    if (n_pix > 0 && (!offsets || !feat2d || !accum)) return fail(ctx, DV_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e = dv::feat_fuse(n_pix, offsets, voxel, weight, feat2d, C, accum, wsum, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "feature fusion");
    return DV_OK;
}

// ---- LiDAR-guided initialisation (Sec. 3.3) ----

static dv_status init_begin(dv_ctx* ctx, const uint64_t* keys, int64_t n, int32_t max_level, dv::Arena& ar,
                            cudaStream_t s) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n < 0 || (n > 0 && !keys)) return fail(ctx, DV_ERR_INVALID_ARG, "bad key array");
    if (n > ((int64_t)1 << 28)) return fail(ctx, DV_ERR_CAPACITY, "more than 2^28 leaves");
    if (max_level < 0 || max_level > 18) return fail(ctx, DV_ERR_INVALID_ARG, "max_level out of range (0..18)");
    uint32_t lv = 0;
    cudaError_t e = dv::key_levels(keys, n, &lv, ar, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "key levels");
    if (lv >> (max_level + 1)) return fail(ctx, DV_ERR_INVALID_ARG, "a leaf level above max_level");
    return DV_OK;
}

dv_status dv_shared_corners(dv_ctx* ctx, const uint64_t* keys, int64_t n, int32_t max_level, uint64_t* grid,
                            uint32_t* index, int64_t* n_corners, void* stream) {
    if (!n_corners) return DV_ERR_INVALID_ARG;
    *n_corners = 0;
    if (ctx) ctx->err.clear();
    if (n > 0 && (!grid || !index)) return fail(ctx, DV_ERR_INVALID_ARG, "NULL output");
    DeviceGuard g(ctx ? ctx->device : 0);
    cudaStream_t s = (cudaStream_t)stream;
    dv::Arena ar;
    ar.pool = ctx ? ctx->pool : nullptr;
    ar.stream = s;
    dv_status st = init_begin(ctx, keys, n, max_level, ar, s);
    cudaError_t e = cudaSuccess;
    bool timeout = false;
    if (st == DV_OK) e = dv::shared_corners(keys, n, max_level, grid, index, n_corners, ar, s, &timeout);
    ar.release();
    if (st != DV_OK) return st;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "shared corners");
    if (timeout) return fail(ctx, DV_ERR_TIMEOUT, "the corner sort ran out of its bounded wait; output invalid");
    return DV_OK;
}

dv_status dv_soft_prior(dv_ctx* ctx, const uint64_t* grid, int64_t n_corners, const double* center, double root_size,
                        int32_t max_level, const float* cloud, int64_t n_points, float s_min, float v_close,
                        float v_far, float* dens, void* stream) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n_corners < 0 || n_points < 0 || !center || !(root_size > 0.0) || !(s_min > 0.0f) || max_level < 0 ||
        max_level > 18 || n_points > ((int64_t)1 << 31))
        return fail(ctx, DV_ERR_INVALID_ARG, "bad arguments");
    if ((n_corners > 0 && (!grid || !dens)) || (n_points > 0 && !cloud))
        return fail(ctx, DV_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    dv::Arena ar;
    ar.pool = ctx->pool;
    ar.stream = s;
    bool timeout = false;
    cudaError_t e = dv::soft_prior(grid, n_corners, center, root_size, max_level, cloud, n_points, s_min, v_close, v_far,
                                   dens, ar, s, &timeout);
    ar.release();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "soft prior");
    if (timeout) return fail(ctx, DV_ERR_TIMEOUT, "the point-cell sort ran out of its bounded wait; output invalid");
    return DV_OK;
}

dv_status dv_subdivide_round(dv_ctx* ctx, const uint64_t* keys, int64_t n, int32_t max_level, const double* center,
                             double root_size, const float* cloud, int64_t n_points, float threshold, uint64_t* out,
                             int64_t* n_out, void* stream) {
    if (!n_out) return DV_ERR_INVALID_ARG;
    *n_out = 0;
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!center || !(root_size > 0.0) || !(threshold >= 0.0f) || n_points < 0 || (n_points > 0 && !cloud) ||
        (n > 0 && !out) || max_level >= 18)
        return fail(ctx, DV_ERR_INVALID_ARG, "bad arguments (children must stay within level 18)");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    dv::Arena ar;
    ar.pool = ctx->pool;
    ar.stream = s;
    dv_status st = init_begin(ctx, keys, n, max_level, ar, s);
    cudaError_t e = cudaSuccess;
    bool timeout = false;
    if (st == DV_OK)
        e = dv::subdivide_round(keys, n, center, root_size, max_level, cloud, n_points, threshold, out, n_out, ar, s,
                                &timeout);
    ar.release();
    if (st != DV_OK) return st;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "subdivision");
    if (timeout) {
        *n_out = 0;
        return fail(ctx, DV_ERR_TIMEOUT, "the leaf-key sort ran out of its bounded wait; nothing was written");
    }
    return DV_OK;
}

dv_status dv_visibility_prune(dv_ctx* ctx, const uint64_t* keys, int64_t n, int32_t max_level, const double* center,
                              double root_size, const dv_camera* cams, int32_t n_cam, double z_min, uint64_t* out,
                              int64_t* n_out, void* stream) {
    if (!n_out) return DV_ERR_INVALID_ARG;
    *n_out = 0;
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!center || !(root_size > 0.0) || n_cam < 0 || n_cam > DV_MAX_VIEWS || (n_cam > 0 && !cams) ||
        (n > 0 && !out))
        return fail(ctx, DV_ERR_INVALID_ARG, "bad arguments");
    std::vector<dv::InitCam> ic((size_t)std::max(n_cam, 1));
    for (int c = 0; c < n_cam; ++c) {
        const dv_camera& cm = cams[c];
        if (cm.W < 0 || cm.H < 0 || !(cm.fx > 0.0f) || !(cm.fy > 0.0f) || !(cm.near_ > 0.0f) || !(cm.far_ > cm.near_))
            return fail(ctx, DV_ERR_INVALID_ARG, "bad camera");
        for (int k = 0; k < 9; ++k) ic[c].R[k] = cm.cam_to_world.R[k];
        for (int k = 0; k < 3; ++k) ic[c].t[k] = cm.cam_to_world.t[k];
        ic[c].fx = cm.fx;
        ic[c].fy = cm.fy;
        ic[c].cx = cm.cx;
        ic[c].cy = cm.cy;
        ic[c].near_ = cm.near_;
        ic[c].far_ = cm.far_;
        ic[c].W = cm.W;
        ic[c].H = cm.H;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    dv::Arena ar;
    ar.pool = ctx->pool;
    ar.stream = s;
    dv_status st = init_begin(ctx, keys, n, max_level, ar, s);
    cudaError_t e = cudaSuccess;
    if (st == DV_OK)
        e = dv::visibility_prune(keys, n, center, root_size, ic.data(), n_cam, z_min, out, n_out, ar, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the camera array is read from host memory
    ar.release();
    if (st != DV_OK) return st;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "visibility pruning");
    return DV_OK;
}

dv_status dv_corner_gather(dv_ctx* ctx, const uint32_t* index, int64_t n, const float* corner, float* dens,
                           void* stream) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n < 0 || (n > 0 && (!index || !corner || !dens))) return fail(ctx, DV_ERR_INVALID_ARG, "bad arguments");
    DeviceGuard g(ctx->device);
    cudaError_t e = dv::corner_gather(index, n, corner, dens, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "corner gather");
    return DV_OK;
}

dv_status dv_corner_scatter(dv_ctx* ctx, const uint32_t* index, int64_t n, const float* d_dens, float* d_corner,
                            void* stream) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n < 0 || (n > 0 && (!index || !d_dens || !d_corner))) return fail(ctx, DV_ERR_INVALID_ARG, "bad arguments");
    DeviceGuard g(ctx->device);
    cudaError_t e = dv::corner_scatter(index, n, d_dens, d_corner, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "corner scatter");
    return DV_OK;
}

// ---- sky composite (Eq. 2) ----

static dv_status sky_views(dv_ctx* ctx, const dv_camera* cams, int32_t n_cam, int32_t env_h, int32_t env_w,
                           std::vector<dv::SkyView>& out) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n_cam < 0 || n_cam > DV_MAX_VIEWS || (n_cam > 0 && !cams))
        return fail(ctx, n_cam > DV_MAX_VIEWS ? DV_ERR_CAPACITY : DV_ERR_INVALID_ARG, "bad camera array");
    if (env_h < 1 || env_w < 1 || (int64_t)env_h * env_w > ((int64_t)1 << 28))
        return fail(ctx, DV_ERR_INVALID_ARG, "environment map size out of range");
    out.resize((size_t)n_cam);
    for (int v = 0; v < n_cam; ++v) {
        const dv_camera& c = cams[v];
        if (c.W < 0 || c.H < 0 || c.W > DV_MAX_IMAGE || c.H > DV_MAX_IMAGE || !(c.fx > 0.0f) || !(c.fy > 0.0f) ||
            !std::isfinite(c.cx) || !std::isfinite(c.cy))
            return fail(ctx, DV_ERR_INVALID_ARG, "bad camera");
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(c.cam_to_world.R[k])) return fail(ctx, DV_ERR_INVALID_POSE, "bad camera rotation");
        dv::SkyView& s = out[v];
        for (int k = 0; k < 9; ++k) s.R[k] = c.cam_to_world.R[k];
        s.fx = c.fx;
        s.fy = c.fy;
        s.cx = c.cx;
        s.cy = c.cy;
        s.W = c.W;
        s.H = c.H;
    }
    return DV_OK;
}

dv_status dv_sky_composite(dv_ctx* ctx, const dv_camera* cams, int32_t n_cam, const float* env, int32_t env_h,
                           int32_t env_w, const float* rgb, const float* alpha, float* out, void* stream) {
    std::vector<dv::SkyView> vs;
    dv_status st = sky_views(ctx, cams, n_cam, env_h, env_w, vs);
    if (st != DV_OK) return st;
    int64_t pix = 0;
    for (auto& v : vs) pix += (int64_t)v.W * v.H;
    if (pix > 0 && (!env || !rgb || !alpha || !out)) return fail(ctx, DV_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int64_t off = 0;
    for (auto& v : vs) {
        cudaError_t e = dv::launch_sky_fwd(v, env, env_h, env_w, rgb + off * 3, alpha + off, out + off * 3, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sky composite");
        off += (int64_t)v.W * v.H;
    }
    return DV_OK;
}

dv_status dv_sky_backward(dv_ctx* ctx, const dv_camera* cams, int32_t n_cam, const float* env, int32_t env_h,
                          int32_t env_w, const float* alpha, const float* d_out, float* d_env, float* d_alpha,
                          void* stream) {
    std::vector<dv::SkyView> vs;
    dv_status st = sky_views(ctx, cams, n_cam, env_h, env_w, vs);
    if (st != DV_OK) return st;
    int64_t pix = 0;
    for (auto& v : vs) pix += (int64_t)v.W * v.H;
    if (pix > 0 && (!env || !alpha || !d_out)) return fail(ctx, DV_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int64_t off = 0;
    for (auto& v : vs) {
        cudaError_t e = dv::launch_sky_bwd(v, env, env_h, env_w, alpha + off, d_out + off * 3, d_env,
                                           d_alpha ? d_alpha + off : nullptr, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sky backward");
        off += (int64_t)v.W * v.H;
    }
    return DV_OK;
}

dv_status dv_state_stats(const dv_state* st, int32_t view, int64_t* n_visible, int64_t* n_pairs, int64_t* n_tiles) {
    if (!st) return DV_ERR_INVALID_ARG;
    const BatchState& B = st->b;
    if (view == -1 || (view == 0 && B.bp.n_view == 1)) {
        if (n_visible) *n_visible = B.n_vis;
        if (n_pairs) *n_pairs = B.n_pairs;
        if (n_tiles) *n_tiles = B.bp.n_tiles;
        return DV_OK;
    }
    if (view < 0 || view >= B.bp.n_view) return DV_ERR_INVALID_ARG;
    DeviceGuard g(st->ctx->device);
    const int n_oct = B.bp.n_oct;
    uint32_t vs[2] = {0, 0};
    const int t0 = B.bp.tile_base[view], t1 = B.bp.tile_base[view + 1];
    cudaError_t e = cudaMemcpyAsync(&vs[0], B.vis_start + (size_t)view * n_oct, 4, cudaMemcpyDeviceToHost, st->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&vs[1], B.vis_start + (size_t)(view + 1) * n_oct, 4, cudaMemcpyDeviceToHost, st->stream);
    // pairs of the view: from the first tile's start to the last tile's end (tiles are contiguous per view)
    std::vector<uint2> rg((size_t)(t1 - t0));
    if (e == cudaSuccess && t1 > t0)
        e = cudaMemcpyAsync(rg.data(), B.range + t0, sizeof(uint2) * rg.size(), cudaMemcpyDeviceToHost, st->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) return DV_ERR_CUDA;
    int64_t np = 0;
    for (const uint2& x : rg) np += (int64_t)x.y - (int64_t)x.x;
    if (n_visible) *n_visible = (int64_t)vs[1] - (int64_t)vs[0];
    if (n_pairs) *n_pairs = np;
    if (n_tiles) *n_tiles = t1 - t0;
    return DV_OK;
}

dv_status dv_state_work(const dv_state* st, int32_t view, uint64_t* tests, uint64_t* box_tests, uint64_t* segments) {
    if (!st) return DV_ERR_INVALID_ARG;
    const BatchState& B = st->b;
    if (!(view == -1 || (view == 0 && B.bp.n_view == 1))) return DV_ERR_INVALID_ARG;
    unsigned long long h[4] = {0, 0, 0, 0};
    if (B.work) {
        DeviceGuard g(st->ctx->device);
        if (cudaMemcpyAsync(h, B.work, sizeof(h), cudaMemcpyDeviceToHost, st->stream) != cudaSuccess ||
            cudaStreamSynchronize(st->stream) != cudaSuccess)
            return DV_ERR_CUDA;
    }
    if (tests) *tests = h[0];
    if (box_tests) *box_tests = h[1];
    if (segments) *segments = h[2];
    return DV_OK;
}

long long dv_launch_count(int32_t reset) {
    return reset ? g_launches.exchange(0) : g_launches.load();
}

dv_status dv_state_check(const dv_state* st, int32_t wait) {
    if (!st) return DV_ERR_INVALID_ARG;
    uint64_t f = state_sort_flag(st);
    if (f == kStatusPending && wait) {
        DeviceGuard g(st->ctx->device);
        if (cudaStreamSynchronize(st->stream) != cudaSuccess) return DV_ERR_CUDA;
        f = state_sort_flag(st);
    }
    return f == 1 ? DV_ERR_TIMEOUT : DV_OK;
}

dv_status dv_debug_sort_timeout(dv_ctx* ctx, int32_t spin_limit, uint32_t* call_flag, uint32_t* device_flag) {
    if (!ctx || !call_flag || !device_flag || spin_limit < 1 || spin_limit > (1 << 20)) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    DeviceGuard g(ctx->device);
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = dv::debug_sort_timeout(spin_limit, call_flag, device_flag, s);
    if (s) cudaStreamDestroy(s);
    return e == cudaSuccess ? DV_OK : cuda_fail(ctx, e, "debug sort timeout");
}

dv_status dv_reserve(dv_ctx* ctx, int64_t bytes) {
    if (!ctx || bytes < 0) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    ctx->budget = bytes;
    if (bytes == 0) return DV_OK;
    // grow the pool to the reservation now (it keeps freed memory: release threshold unlimited), so
    // the calls within it take their workspace without new device allocations
    DeviceGuard g(ctx->device);
    cudaStream_t s = nullptr;
    void* p = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&p, (size_t)bytes, ctx->pool, s);
    if (e == cudaSuccess) e = cudaFreeAsync(p, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (s) cudaStreamDestroy(s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        ctx->budget = 0;
        return fail(ctx, DV_ERR_NOMEM, "the device cannot hold a reservation of " + std::to_string(bytes) + " bytes");
    }
    return e == cudaSuccess ? DV_OK : cuda_fail(ctx, e, "reserve");
}

dv_status dv_workspace_need(const dv_ctx* ctx, int64_t* bytes) {
    if (!ctx || !bytes) return DV_ERR_INVALID_ARG;
    *bytes = ctx->last_need;
    return DV_OK;
}

dv_status dv_asset_init(dv_ctx* ctx, const float* box_dims, int32_t level, float v_init, int64_t capacity,
                        uint64_t* keys, float* dens, double* root_size, int64_t* n_leaves, void* stream) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!box_dims || !root_size || !n_leaves) return fail(ctx, DV_ERR_INVALID_ARG, "NULL argument");
    *n_leaves = 0;
    *root_size = 0.0;
    double m = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (!(box_dims[k] > 0.0f) || !std::isfinite(box_dims[k]))
            return fail(ctx, DV_ERR_INVALID_ARG, "box dimensions must be finite and > 0");
        m = std::max(m, (double)box_dims[k]);
    }
    if (level < 0 || level > 10) return fail(ctx, DV_ERR_INVALID_ARG, "level out of range (0..10)");
    if (!std::isfinite(v_init)) return fail(ctx, DV_ERR_INVALID_ARG, "non-finite initial density");
    const int64_t n = (int64_t)1 << (3 * level);
    if (capacity < n)
        return fail(ctx, DV_ERR_CAPACITY, "the grid has " + std::to_string(n) + " leaves, above the capacity of " +
                                              std::to_string(capacity));
    if (!keys || !dens) return fail(ctx, DV_ERR_INVALID_ARG, "NULL output buffer");
    if ((uintptr_t)dens & 15) return fail(ctx, DV_ERR_INVALID_ARG, "dens must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    const cudaError_t e = dv::asset_grid(level, v_init, keys, dens, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "asset grid");
    *root_size = 1.2 * m;
    *n_leaves = n;
    return DV_OK;
}

dv_status dv_profile_enable(dv_ctx* ctx, int32_t on) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->profiling = on != 0;
    ctx->prof_mask = ~0u;
    return DV_OK;
}

dv_status dv_profile_enable_stages(dv_ctx* ctx, uint32_t mask) {
    if (!ctx) return DV_ERR_INVALID_ARG;
    ctx->profiling = mask != 0;
    ctx->prof_mask = mask;
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

namespace dv {
// Camera and pose checks of one render request (the serving loop's admission).
dv_status validate_request(const dv_camera& cam, const dv_pose* poses, int n_oct) {
    return validate_view(nullptr, cam, poses, n_oct);
}

// Render of views whose outputs live in separate buffers (used by the serving loop).
dv_status render_views_into(dv_ctx* ctx, const dv_octree* oct, int n_oct, const dv_view* views, int n_view,
                            const dv_opts* opts, float* const* rgbs, float* const* depths, float* const* alphas,
                            dv_state** saved, void* stream) {
    std::vector<const dv_pose*> vp((size_t)std::max(n_view, 1), nullptr);
    std::vector<dv_camera> cams((size_t)std::max(n_view, 1));
    for (int v = 0; v < n_view; ++v) {
        vp[v] = views[v].poses;
        cams[v] = views[v].camera;
    }
    return render_common(ctx, oct, n_oct, vp.data(), cams.data(), n_view, opts, nullptr, nullptr, nullptr, rgbs, depths,
                         alphas, saved, stream);
}
}  // namespace dv

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
//  * at most DV_STATIC_MAX_VISIBLE visible voxels per render call, summed over
//    its views (12 floats each, 6 MiB in total); a larger call is rejected
//    with DV_ERR_CAPACITY before any work is enqueued;
//  * every GPU that loads this library holds the array until the process exits;
//  * all calls on a device share the one array: the slice a call uses is cleared
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
    if (st->b.n_vis > DV_STATIC_MAX_VISIBLE)
        return fail(ctx, DV_ERR_CAPACITY,
                    "dv_render_backward_static: the render call has " + std::to_string(st->b.n_vis) +
                        " visible voxels, above the static limit of " + std::to_string(DV_STATIC_MAX_VISIBLE));
    if (st->b.n_vis == 0) return DV_OK;
    DeviceGuard g(ctx->device);
    float* grad = nullptr;
    cudaError_t e = static_grad_ptr(ctx->device, &grad);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(static gradient scratch)");
    return backward_batch(ctx, st, d_rgb, d_depth, d_alpha, nullptr, d_dens, d_sh, grad, (cudaStream_t)stream);
}
