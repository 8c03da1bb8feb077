// Continuous-batching render server.
//
// Requests (a camera plus the pose of every octree at the request's timestamp,
// and caller-owned device output buffers) enter a FIFO queue.  Worker threads,
// each with its own CUDA stream and library context, take as many queued
// requests as the admission limits allow (views per batch, pixels per batch,
// pixels rendering at once over all workers -- the device-memory budget), render
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

#include <atomic>
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
    int64_t next_ticket = 1;
    int64_t inflight_pixels = 0;
    int64_t n_batches = 0, n_views = 0, max_batch = 0;
    std::string err;
};

namespace {

void worker_loop(dv_server* S, int k) {
    cudaSetDevice(S->device);
    dv_ctx* ctx = S->ctxs[k];
    cudaStream_t stream = S->streams[k];
    const int n_oct = (int)S->oct.size();
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        int64_t pixels = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                if (S->stop && S->queue.empty()) return true;
                if (S->queue.empty()) return false;
                const int64_t p = S->queue.front()->pixels;
                return S->inflight_pixels == 0 || S->inflight_pixels + p <= S->cfg.max_inflight_pixels;
            });
            if (S->stop && S->queue.empty()) return;
            while (!S->queue.empty() && (int)batch.size() < S->cfg.max_views) {
                const int64_t p = S->queue.front()->pixels;
                if (!batch.empty() && pixels + p > S->cfg.max_batch_pixels) break;
                if (S->inflight_pixels + pixels > 0 && S->inflight_pixels + pixels + p > S->cfg.max_inflight_pixels)
                    break;
                batch.push_back(S->queue.front());
                S->queue.pop_front();
                pixels += p;
            }
            if (batch.empty()) continue;
            S->inflight_pixels += pixels;
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
        dv_status st = dv::render_views_into(ctx, S->oct.data(), n_oct, views.data(), (int)views.size(), &S->cfg.opts,
                                             rgbs.data(), depths.data(), alphas.data(), stream);
        std::string msg = st == DV_OK ? "" : dv_last_error(ctx);
        if (st == DV_OK && cudaStreamSynchronize(stream) != cudaSuccess) {
            st = DV_ERR_CUDA;
            msg = "stream synchronisation failed";
        }
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
        cfg->max_batch_pixels < 1 || cfg->max_inflight_pixels < 1)
        return DV_ERR_INVALID_ARG;
    std::unique_ptr<dv_server> S(new (std::nothrow) dv_server());
    if (!S) return DV_ERR_NOMEM;
    S->device = device;
    S->oct.assign(oct, oct + n_oct);
    S->cfg = *cfg;
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
