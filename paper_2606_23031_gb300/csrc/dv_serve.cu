// Continuous-batching render server.
//
// Requests (a camera plus the pose of every octree at the request's timestamp,
// and caller-owned device output buffers) enter a FIFO queue.  Worker threads,
// each with its own CUDA stream and library context, take as many queued
// requests as the admission limits allow (views per batch, pixels per batch,
// pixels rendering at once over all workers, and the device memory the batches
// in flight take from the library's pools), render
// them as one batch of views (one launch per stage for all of them, tiles of
// every request scheduled together), wait for the batch's stream, and mark the
// requests done.  Requests that arrive while batches are on the GPU join the
// next batch that a worker forms; with several workers the batches overlap on
// the device.  The scene octrees stay resident (borrowed device buffers).
//
// All waits are host-side and bounded by the caller (dv_serve_wait); no kernel
// waits on another.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dv.h"
#include "dv_internal.cuh"

namespace {

using clock_type = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    dv_camera cam{};
    std::vector<dv_pose> poses;
    float* rgb = nullptr;
    float* depth = nullptr;
    float* alpha = nullptr;
    int64_t pixels = 0;
    int64_t bytes = 0;  // device memory estimated at admission
    clock_type::time_point t_submit;
    clock_type::time_point t_done;
    dv_status status = DV_OK;
    bool done = false;
};

}  // namespace

struct dv_server {
    int device = 0;
    std::vector<dv_octree> oct;
    dv_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work;  // queue or budget changed
    std::condition_variable cv_done;  // a batch finished
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Request>> live;
    std::vector<std::thread> workers;
    std::vector<dv_ctx*> ctxs;
    std::vector<cudaStream_t> streams;
    bool stop = false;
    bool paused = false;
    int64_t next_ticket = 1;
    int64_t inflight_pixels = 0;
    int64_t inflight_bytes = 0, peak_inflight_bytes = 0, last_request_bytes = 0;
    int64_t n_batches = 0, n_views = 0, max_batch = 0;
    // device-memory model of a request: the visible fraction of the scene's voxels per view (it does
    // not depend on the resolution) and the (tile, voxel) pairs per tile (a voxel covers more tiles at
    // a higher resolution), running estimates from the finished batches (the first batch uses the
    // conservative starting values)
    double vis_frac = 1.0, pairs_per_tile = 256.0;
    int64_t n_vox = 0;
    int key_bits = 64;
    std::string err;
};

namespace {

int bits_of(int64_t n) {
    int b = 0;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

// device memory a request will take while it renders, from the running model (S->mu held): the part
// its size fixes (the per-voxel projection arrays, per-pixel and per-tile state) plus the estimated
// visible voxels and pairs, with a 25% margin
int64_t request_bytes(const dv_server* S, const Request& r) {
    const int64_t tiles = (int64_t)((r.cam.W + 15) / 16) * ((r.cam.H + 15) / 16);
    const int64_t n_vis = (int64_t)std::ceil(S->vis_frac * (double)S->n_vox);
    const int64_t P = (int64_t)std::ceil(S->pairs_per_tile * (double)tiles);
    const int64_t b = dv::render_need_before(1, (int64_t)S->oct.size(), S->n_vox, tiles, r.pixels) +
                      dv::render_need_after(n_vis, P, tiles, S->key_bits, bits_of(std::max<int64_t>(tiles, 2)), false);
    return b + b / 4;
}

void worker_loop(dv_server* S, int k) {
    cudaSetDevice(S->device);
    dv_ctx* ctx = S->ctxs[k];
    cudaStream_t stream = S->streams[k];
    const int n_oct = (int)S->oct.size();
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        int64_t pixels = 0, bytes = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // a request is admitted when its pixels and its device memory fit beside the batches in
            // flight (or when nothing is in flight: a request larger than the budget runs alone)
            auto fits = [&](const Request& r, int64_t px_more, int64_t by_more) {
                const int64_t px = S->inflight_pixels + px_more, by = S->inflight_bytes + by_more;
                if (px + by == 0) return true;
                if (px + r.pixels > S->cfg.max_inflight_pixels) return false;
                return S->cfg.max_inflight_bytes <= 0 || by + request_bytes(S, r) <= S->cfg.max_inflight_bytes;
            };
            S->cv_work.wait(lk, [&] {
                if (S->stop && S->queue.empty()) return true;
                if (S->queue.empty() || (S->paused && !S->stop)) return false;
                return fits(*S->queue.front(), 0, 0);
            });
            if (S->stop && S->queue.empty()) return;
            while (!S->queue.empty() && (int)batch.size() < S->cfg.max_views) {
                Request& r = *S->queue.front();
                if (!batch.empty() && pixels + r.pixels > S->cfg.max_batch_pixels) break;
                if (!fits(r, pixels, bytes)) break;
                r.bytes = request_bytes(S, r);
                S->last_request_bytes = r.bytes;
                batch.push_back(S->queue.front());
                S->queue.pop_front();
                pixels += r.pixels;
                bytes += r.bytes;
            }
            if (batch.empty()) continue;
            S->inflight_pixels += pixels;
            S->inflight_bytes += bytes;
            S->peak_inflight_bytes = std::max(S->peak_inflight_bytes, S->inflight_bytes);
        }
        std::vector<dv_view> views(batch.size());
        std::vector<float*> rgbs(batch.size()), depths(batch.size()), alphas(batch.size());
        for (size_t i = 0; i < batch.size(); ++i) {
            views[i].camera = batch[i]->cam;
            views[i].poses = batch[i]->poses.data();
            rgbs[i] = batch[i]->rgb;
            depths[i] = batch[i]->depth;
            alphas[i] = batch[i]->alpha;
        }
        dv_state* state = nullptr;
        dv_status st = dv::render_views_into(ctx, S->oct.data(), n_oct, views.data(), (int)views.size(), &S->cfg.opts,
                                             rgbs.data(), depths.data(), alphas.data(), &state, stream);
        std::string msg = st == DV_OK ? "" : dv_last_error(ctx);
        if (st == DV_OK && cudaStreamSynchronize(stream) != cudaSuccess) {
            st = DV_ERR_CUDA;
            msg = "stream synchronisation failed";
        }
        // the batch's own sorts: a bounded wait that ran out fails this batch's requests
        if (st == DV_OK && dv_state_check(state, 0) == DV_ERR_TIMEOUT) {
            st = DV_ERR_TIMEOUT;
            msg = "a sort of this batch ran out of its bounded wait";
        }
        int64_t n_vis = -1, n_pairs = 0, n_tiles = 0;
        if (st == DV_OK && state) dv_state_stats(state, -1, &n_vis, &n_pairs, &n_tiles);
        dv_state_free(state);
        const clock_type::time_point now = clock_type::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto& r : batch) {
                r->status = st;
                r->t_done = now;
                r->done = true;
            }
            if (st != DV_OK) S->err = msg;
            S->inflight_pixels -= pixels;
            S->inflight_bytes -= bytes;
            if (n_vis >= 0 && S->n_vox > 0) {
                // running estimates of the memory model from what this batch really had
                const double vf = (double)n_vis / ((double)S->n_vox * (double)batch.size());
                const double pt = n_tiles > 0 ? (double)n_pairs / (double)n_tiles : S->pairs_per_tile;
                const bool first = S->n_batches == 0;
                S->vis_frac = first ? vf : 0.7 * S->vis_frac + 0.3 * vf;
                S->pairs_per_tile = first ? pt : 0.7 * S->pairs_per_tile + 0.3 * pt;
            }
            S->n_batches += 1;
            S->n_views += (int64_t)batch.size();
            if ((int64_t)batch.size() > S->max_batch) S->max_batch = (int64_t)batch.size();
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

dv_status dv_serve_create(dv_server** out, int32_t device, const dv_octree* oct, int32_t n_oct,
                          const dv_serve_config* cfg) {
    if (!out) return DV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!oct || n_oct < 1 || n_oct > DV_MAX_OCTREES || !cfg) return DV_ERR_INVALID_ARG;
    if (cfg->max_views < 1 || cfg->max_views > DV_MAX_VIEWS || cfg->n_workers < 1 || cfg->n_workers > 8 ||
        cfg->max_batch_pixels < 1 || cfg->max_inflight_pixels < 1 || cfg->max_inflight_bytes < 0)
        return DV_ERR_INVALID_ARG;
    std::unique_ptr<dv_server> S(new (std::nothrow) dv_server());
    if (!S) return DV_ERR_NOMEM;
    S->device = device;
    S->oct.assign(oct, oct + n_oct);
    S->cfg = *cfg;
    int lkey = 0;
    for (int i = 0; i < n_oct; ++i) {
        S->n_vox += oct[i].n_vox;
        lkey = std::max(lkey, (int)oct[i].max_level);
    }
    S->key_bits = std::min(64, 3 * lkey + bits_of(n_oct) + bits_of(cfg->max_views));
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return DV_ERR_INVALID_ARG;
    for (int k = 0; k < cfg->n_workers; ++k) {
        dv_ctx* c = nullptr;
        dv_status st = dv_create(&c, device);
        cudaStream_t s = nullptr;
        if (st == DV_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = DV_ERR_CUDA;
        if (st != DV_OK) {
            if (c) dv_destroy(c);
            for (auto x : S->ctxs) dv_destroy(x);
            for (auto x : S->streams) cudaStreamDestroy(x);
            if (prev >= 0) cudaSetDevice(prev);
            return st;
        }
        S->ctxs.push_back(c);
        S->streams.push_back(s);
    }
    if (prev >= 0) cudaSetDevice(prev);
    dv_server* raw = S.get();
    for (int k = 0; k < cfg->n_workers; ++k) S->workers.emplace_back(worker_loop, raw, k);
    *out = S.release();
    return DV_OK;
}

dv_status dv_serve_submit(dv_server* S, const dv_camera* cam, const dv_pose* poses, float* rgb, float* depth,
                          float* alpha, int64_t* ticket) {
    if (!S || !cam || !poses || !ticket) return DV_ERR_INVALID_ARG;
    const int64_t px = (int64_t)cam->W * cam->H;
    if (cam->W < 0 || cam->H < 0 || (px > 0 && (!rgb || !depth || !alpha))) return DV_ERR_INVALID_ARG;
    // a request that would fail its render (non-finite or non-rigid pose, bad intrinsics) is rejected
    // here, before it can join a batch and fail the requests batched with it
    const dv_status vs = dv::validate_request(*cam, poses, (int)S->oct.size());
    if (vs != DV_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "request rejected at admission (bad camera or pose)";
        return vs;
    }
    auto r = std::make_shared<Request>();
    r->cam = *cam;
    r->poses.assign(poses, poses + S->oct.size());
    r->rgb = rgb;
    r->depth = depth;
    r->alpha = alpha;
    r->pixels = px;
    r->t_submit = clock_type::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return DV_ERR_INVALID_ARG;
        r->ticket = S->next_ticket++;
        S->live[r->ticket] = r;
        S->queue.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_one();
    return DV_OK;
}

static double latency_ms(const Request& r) {
    return std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
}

dv_status dv_serve_poll(dv_server* S, int64_t ticket, int32_t* done, double* lat_ms) {
    if (!S || !done) return DV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end()) return DV_ERR_INVALID_ARG;
    *done = it->second->done ? 1 : 0;
    if (it->second->done) {
        if (lat_ms) *lat_ms = latency_ms(*it->second);
        return it->second->status;
    }
    return DV_OK;
}

dv_status dv_serve_wait(dv_server* S, int64_t ticket, double timeout_ms, double* lat_ms) {
    if (!S) return DV_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end()) return DV_ERR_INVALID_ARG;
    std::shared_ptr<Request> r = it->second;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                        [&] { return r->done; });
    if (!ok) return DV_ERR_TIMEOUT;
    if (lat_ms) *lat_ms = latency_ms(*r);
    return r->status;
}

dv_status dv_serve_release(dv_server* S, int64_t ticket) {
    if (!S) return DV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end() || !it->second->done) return DV_ERR_INVALID_ARG;
    S->live.erase(it);
    return DV_OK;
}

dv_status dv_serve_pause(dv_server* S, int32_t paused) {
    if (!S) return DV_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->paused = paused != 0;
    }
    S->cv_work.notify_all();
    return DV_OK;
}

dv_status dv_serve_memory(dv_server* S, int32_t reset_peak, int64_t* inflight_bytes, int64_t* peak_inflight_bytes,
                          int64_t* last_request_bytes) {
    if (!S) return DV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (inflight_bytes) *inflight_bytes = S->inflight_bytes;
    if (peak_inflight_bytes) *peak_inflight_bytes = S->peak_inflight_bytes;
    if (last_request_bytes) *last_request_bytes = S->last_request_bytes;
    if (reset_peak) S->peak_inflight_bytes = S->inflight_bytes;
    return DV_OK;
}

dv_status dv_serve_stats(dv_server* S, int64_t* batches, int64_t* views, int64_t* max_batch) {
    if (!S) return DV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (batches) *batches = S->n_batches;
    if (views) *views = S->n_views;
    if (max_batch) *max_batch = S->max_batch;
    return DV_OK;
}

const char* dv_serve_last_error(const dv_server* S) { return S ? S->err.c_str() : "no server"; }

void dv_serve_destroy(dv_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers)
        if (t.joinable()) t.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto c : S->ctxs) dv_destroy(c);
    for (auto s : S->streams) cudaStreamDestroy(s);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
