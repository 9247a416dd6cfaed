// occ_server.cu -- the serving loop of include/occ_serve.h: a native worker thread that
// admits requests with the scheduler (occ_sched.cpp), runs each admitted batch on its own
// stream and context (G-buffer, trace, reuse, result copy), and reports per-request
// timestamps.  Device memory comes from a stream-ordered pool owned by the server.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "occ_internal.h"
#include "occ_sched.h"
#include "occ_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t kAlign = 256;

int64_t align_up(int64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Req {
    occ_request r;
    std::vector<int32_t> offsets;   // copy of the pattern's offsets
    int64_t bytes = 0;
    int64_t t_submit = 0, t_admit = 0;
    char* mem = nullptr;            // one pool allocation, carved below
    float* pos = nullptr;
    float* nrm = nullptr;
    void* rec = nullptr;
    float* out = nullptr;
};

// Device bytes of one request: G-buffer, records and (unless the caller gives a device
// output) the estimate, each plane 256-byte aligned.
int64_t request_bytes(const occ_request& r) {
    const int64_t P = (int64_t)r.W * r.H;
    const int64_t plane = 16 * P;
    int64_t b = align_up(plane);                        // pos4 / packed plane
    if (!r.packed) b += align_up(plane);                // nrm4
    b += r.packed ? align_up(plane) : 2 * align_up(plane);   // records
    if (!r.out_device) b += align_up(4 * P);
    return b;
}

struct Slot {
    cudaStream_t stream = nullptr;
    occ_ctx* ctx = nullptr;
    cudaEvent_t done = nullptr;
    unsigned* status_host = nullptr;   // pinned copy of the context's device status word
    std::vector<uint64_t> ids;
    bool busy = false;
    occ_status launch_status = OCC_OK;
};

}  // namespace

struct occ_server {
    int device = 0;
    const occ_bvh* bvh = nullptr;
    occ_server_config cfg{};
    occ::Tuning tune;
    cudaMemPool_t pool = nullptr;
    occ::Scheduler* sched = nullptr;
    occ_ctx* submit_ctx = nullptr;     // argument checks of submit (under mu)
    std::mutex mu;
    std::mutex join_mu;                // serialises shutdown calls
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<occ_result> done;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false, cancel = false, worker_exited = false;
    uint64_t next_id = 1;
    Clock::time_point t0;
    int64_t batches = 0, views_batched = 0, views_single = 0;
    int32_t inject_left = 0;           // allocation failures still to inject (worker only)

    int64_t now() const {
        return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
    }
};

namespace {

void push_result(occ_server* S, uint64_t id, occ_status st, int views, int64_t t_done) {
    auto it = S->reqs.find(id);
    occ_result res{};
    res.id = id;
    res.status = st;
    res.batch_views = views;
    res.t_done_ns = t_done;
    if (it != S->reqs.end()) {
        res.t_submit_ns = it->second.t_submit;
        res.t_admit_ns = it->second.t_admit;
        S->reqs.erase(it);
    }
    S->done.push_back(res);
}

// Enqueues one batch on the slot's stream.  Runs without the server lock; the requests
// are not touched by other threads while they run.
occ_status launch_batch(occ_server* S, Slot& sl, const std::vector<Req*>& rs) {
    const cudaStream_t s = sl.stream;
    occ_ctx* ctx = sl.ctx;
    occ_status st = OCC_OK;
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return OCC_ERR_CUDA;
    size_t allocated = 0;
    if (S->inject_left > 0) {
        --S->inject_left;   // injected fault: the pool has no room for this batch
        return OCC_ERR_OOM;
    }
    for (Req* q : rs) {
        e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&q->mem), (size_t)q->bytes, S->pool, s);
        if (e != cudaSuccess) {
            st = e == cudaErrorMemoryAllocation ? OCC_ERR_OOM : OCC_ERR_CUDA;
            break;
        }
        ++allocated;
        const occ_request& r = q->r;
        const int64_t P = (int64_t)r.W * r.H, plane = align_up(16 * P);
        char* m = q->mem;
        q->pos = reinterpret_cast<float*>(m);
        m += plane;
        q->nrm = nullptr;
        if (!r.packed) {
            q->nrm = reinterpret_cast<float*>(m);
            m += plane;
        }
        q->rec = m;
        m += r.packed ? plane : 2 * plane;
        q->out = r.out_device ? r.out_device : reinterpret_cast<float*>(m);
        if (r.pos4_host) {
            e = cudaMemcpyAsync(q->pos, r.pos4_host, (size_t)(16 * P), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && !r.packed)
                e = cudaMemcpyAsync(q->nrm, r.nrm4_host, (size_t)(16 * P), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) st = OCC_ERR_CUDA;
        } else {
            st = occ_gbuffer_pinhole(ctx, S->bvh, r.camera, r.eps, r.W, r.H, q->pos, q->nrm, s);
        }
        if (st != OCC_OK) break;
    }
    // small views: one batched launch pair; large views (or K > 16): per-view kernels
    std::vector<occ_view> views;
    std::vector<Req*> single;
    if (st == OCC_OK) {
        for (Req* q : rs) {
            const occ_request& r = q->r;
            occ_gbuffer gb{r.W, r.H, q->pos, q->nrm, r.packed ? OCC_GB_PACKED : OCC_GB_FP32};
            occ_occluders rec{};
            rec.W = r.W;
            rec.H = r.H;
            rec.format = r.packed ? OCC_REC_PACKED : OCC_REC_FP32;
            rec.data = q->rec;
            if ((int64_t)r.W * r.H <= S->cfg.batch_max_px && r.K <= 16) {
                occ_view v{};
                v.gb = gb;
                v.rec = rec;
                v.effect = r.effect;
                v.radius = r.radius;
                v.light = r.light;
                v.seed = r.seed;
                v.sample = r.sample;
                v.pattern = r.pattern;
                v.K = r.K;
                v.estimator = r.estimator;
                v.out = q->out;
                views.push_back(v);
            } else {
                single.push_back(q);
            }
        }
        if (!views.empty())
            st = occ_frame_batch(ctx, S->bvh, views.data(), (int32_t)views.size(), s);
        for (size_t i = 0; st == OCC_OK && i < single.size(); ++i) {
            const occ_request& r = single[i]->r;
            occ_gbuffer gb{r.W, r.H, single[i]->pos, single[i]->nrm,
                           r.packed ? OCC_GB_PACKED : OCC_GB_FP32};
            occ_occluders rec{};
            rec.W = r.W;
            rec.H = r.H;
            rec.format = r.packed ? OCC_REC_PACKED : OCC_REC_FP32;
            rec.data = single[i]->rec;
            const occ_bvh* vb = r.estimator == OCC_EST_UNBIASED ? S->bvh : nullptr;
            if (r.effect == OCC_EFFECT_AO) {
                st = occ_trace_ao(ctx, &gb, S->bvh, r.radius, r.seed, r.sample, &rec, s);
                if (st == OCC_OK)
                    st = occ_reuse_ao(ctx, &gb, &rec, &r.pattern, r.K, r.estimator, vb,
                                      single[i]->out, s);
            } else {
                st = occ_trace_shadow(ctx, &gb, S->bvh, &r.light, r.seed, r.sample, &rec, s);
                if (st == OCC_OK)
                    st = occ_reuse_shadow(ctx, &gb, &rec, &r.pattern, r.K, r.estimator, vb,
                                          single[i]->out, s);
            }
        }
    }
    if (st == OCC_OK)
        for (Req* q : rs)
            if (q->r.out_host) {
                e = cudaMemcpyAsync(q->r.out_host, q->out, (size_t)q->r.W * q->r.H * sizeof(float),
                                    cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) {
                    st = OCC_ERR_CUDA;
                    break;
                }
            }
    if (st == OCC_OK) {
        e = cudaMemcpyAsync(sl.status_host, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = OCC_ERR_CUDA;
    }
    for (size_t i = 0; i < allocated; ++i) cudaFreeAsync(rs[i]->mem, s);
    e = cudaEventRecord(sl.done, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);   // the batch's own work, already queued, ends by itself
        if (st == OCC_OK) st = OCC_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->batches;
        S->views_batched += (int64_t)views.size();
        S->views_single += (int64_t)single.size();
    }
    return st;
}

void worker_main(occ_server* S) {
    cudaSetDevice(S->device);
    std::vector<uint64_t> ids, expired;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool any_done = false, any_busy = false;
        // retire finished batches
        for (size_t i = 0; i < S->slots.size(); ++i) {
            Slot& sl = S->slots[i];
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            const int64_t t = S->now();
            occ_status st = sl.launch_status;
            if (st == OCC_OK && q != cudaSuccess) st = OCC_ERR_CUDA;
            if (st == OCC_OK && *sl.status_host) st = OCC_ERR_DEVICE_CHECK;
            for (uint64_t id : sl.ids) push_result(S, id, st, (int)sl.ids.size(), t);
            S->sched->complete((int)i);
            sl.busy = false;
            sl.ids.clear();
            any_done = true;
        }
        // shutdown with cancellation: queued requests end without running
        if (S->stop && S->cancel) {
            uint64_t buf[256];
            int n;
            while ((n = S->sched->drain(buf, 256)) > 0)
                for (int k = 0; k < n; ++k) push_result(S, buf[k], OCC_ERR_CANCELLED, 0, S->now());
            any_done = true;
        }
        // admission (held while a batching window is open)
        int64_t hold_until = 0;
        if (S->cfg.batch_window_us > 0 && !S->stop) {
            const int64_t q = S->sched->stats().queued;
            if (q > 0 && q < S->cfg.max_views_per_batch) {
                const int64_t due = S->sched->oldest_submit() + 1000 * S->cfg.batch_window_us;
                if (S->now() < due) hold_until = due;
            }
        }
        const int slot = S->sched->next(S->now(), &ids, 256, &expired, 256, hold_until == 0);
        for (uint64_t id : expired) push_result(S, id, OCC_ERR_TIMEOUT, 0, S->now());
        if (any_done || !expired.empty()) S->cv_done.notify_all();
        if (slot >= 0) {
            Slot& sl = S->slots[slot];
            sl.busy = true;
            sl.ids = ids;
            sl.launch_status = OCC_OK;
            std::vector<Req*> rs;
            const int64_t t = S->now();
            for (uint64_t id : ids) {
                Req& r = S->reqs.at(id);
                r.t_admit = t;
                rs.push_back(&r);
            }
            lk.unlock();
            const occ_status st = launch_batch(S, sl, rs);
            lk.lock();
            sl.launch_status = st;
            continue;
        }
        if (!expired.empty()) continue;
        for (const Slot& sl : S->slots) any_busy = any_busy || sl.busy;
        if (S->stop && S->sched->stats().queued == 0 && !any_busy) break;
        if (any_busy) {
            lk.unlock();
            if (S->cfg.poll_us > 0)
                std::this_thread::sleep_for(std::chrono::microseconds(S->cfg.poll_us));
            else
                std::this_thread::yield();
            lk.lock();
        } else if (hold_until > 0) {
            const int64_t q = S->sched->stats().queued;
            S->cv_work.wait_until(lk, S->t0 + std::chrono::nanoseconds(hold_until), [S, q] {
                return S->stop || S->sched->stats().queued != q;
            });
        } else {
            S->cv_work.wait(lk, [S] { return S->stop || S->sched->stats().queued > 0; });
        }
    }
    S->worker_exited = true;
    S->cv_done.notify_all();
}

void release(occ_server* S) {
    cudaSetDevice(S->device);
    for (Slot& sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.status_host) cudaFreeHost(sl.status_host);
        if (sl.ctx) occ_destroy(sl.ctx);
    }
    if (S->pool) cudaMemPoolDestroy(S->pool);
    if (S->submit_ctx) occ_destroy(S->submit_ctx);
    delete S->sched;
    delete S;
}

void set_msg(char* err, int32_t len, const char* msg) {
    if (err && len > 0) {
        std::strncpy(err, msg, (size_t)len - 1);
        err[len - 1] = '\0';
    }
}

bool finite_all(const float* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

OCC_EXPORT occ_status occ_server_create(occ_ctx* ctx, const occ_bvh* bvh,
                                        const occ_server_config* cfg_in, occ_server** out) {
    if (!ctx || !bvh || !out) return OCC_ERR_INVALID_ARG;
    *out = nullptr;
    if (bvh->device != ctx->device) return OCC_ERR_INVALID_ARG;
    occ_server_config cfg = cfg_in ? *cfg_in : occ_server_config{};
    if (cfg.budget_bytes < 0 || cfg.max_views_per_batch < 0 || cfg.max_views_per_batch > 256 ||
        cfg.max_inflight < 0 || cfg.max_inflight > occ::Scheduler::kMaxInflight ||
        cfg.max_queued < 0 || cfg.poll_us < 0 || cfg.batch_max_px < 0 || cfg.batch_window_us < 0 ||
        cfg.inject_alloc_failures < 0)
        return OCC_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return OCC_ERR_CUDA;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return OCC_ERR_CUDA;
    if (cfg.budget_bytes == 0) cfg.budget_bytes = (int64_t)(0.8 * (double)free_b);
    if (cfg.budget_bytes > (int64_t)free_b) return OCC_ERR_OOM;
    if (cfg.max_views_per_batch == 0) cfg.max_views_per_batch = 64;
    if (cfg.max_inflight == 0) cfg.max_inflight = 2;
    if (cfg.max_queued == 0) cfg.max_queued = 4096;
    if (cfg.batch_max_px == 0) cfg.batch_max_px = 1 << 20;

    occ_server* S = new occ_server();
    S->device = ctx->device;
    S->bvh = bvh;
    S->cfg = cfg;
    S->tune = ctx->tune;
    S->inject_left = cfg.inject_alloc_failures;
    S->t0 = Clock::now();
    occ_sched_config sc{cfg.budget_bytes, cfg.max_views_per_batch, cfg.max_inflight, cfg.max_queued};
    S->sched = new occ::Scheduler(sc);
    S->slots.resize(cfg.max_inflight);
    occ_status st = occ_create(S->device, &S->submit_ctx);
    cudaError_t e = cudaSuccess;
    if (st == OCC_OK) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = S->device;
        e = cudaMemPoolCreate(&S->pool, &props);
        uint64_t keep = UINT64_MAX;   // keep freed blocks for the next batch
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (Slot& sl : S->slots) {
        if (st != OCC_OK || e != cudaSuccess) break;
        st = occ_create(S->device, &sl.ctx);
        if (st != OCC_OK) break;
        sl.ctx->tune = S->tune;
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.status_host, sizeof(unsigned));
        if (e == cudaSuccess) *sl.status_host = 0;
    }
    if (st == OCC_OK && e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? OCC_ERR_OOM : OCC_ERR_CUDA;
    if (st != OCC_OK) {
        release(S);
        return st;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_server_submit(occ_server* S, const occ_request* req, uint64_t* id,
                                        char* err_msg, int32_t err_len) {
    if (!S || !req || !id) {
        set_msg(err_msg, err_len, "server, request or id is NULL");
        return OCC_ERR_INVALID_ARG;
    }
    *id = 0;
    const occ_request& r = *req;
    char msg[256];
    auto bad = [&](occ_status st, const char* m) {
        set_msg(err_msg, err_len, m);
        return st;
    };
    if (r.W <= 0 || r.H <= 0 || (int64_t)r.W * r.H > ((int64_t)1 << 31) - 1)
        return bad(OCC_ERR_INVALID_ARG, "request size out of range");
    if (r.effect != OCC_EFFECT_AO && r.effect != OCC_EFFECT_SHADOW)
        return bad(OCC_ERR_INVALID_ARG, "effect invalid");
    if (r.effect == OCC_EFFECT_AO && !(r.radius > 0.0f && std::isfinite(r.radius)))
        return bad(OCC_ERR_INVALID_ARG, "AO radius must be positive and finite");
    if (r.estimator < OCC_EST_NOREUSE || r.estimator > OCC_EST_BOXMEAN)
        return bad(OCC_ERR_INVALID_ARG, "estimator invalid");
    if (r.packed != 0 && r.packed != 1) return bad(OCC_ERR_INVALID_ARG, "packed must be 0 or 1");
    if ((r.out_host == nullptr) == (r.out_device == nullptr))
        return bad(OCC_ERR_INVALID_ARG, "exactly one of out_host and out_device must be set");
    if (r.pos4_host) {
        if (r.packed ? r.nrm4_host != nullptr : r.nrm4_host == nullptr)
            return bad(OCC_ERR_INVALID_ARG, "host G-buffer: FP32 needs nrm4_host, packed takes none");
    } else if (!finite_all(r.camera, 10) || !(r.camera[9] > 0.0f && r.camera[9] < 180.0f) ||
               !std::isfinite(r.eps)) {
        return bad(OCC_ERR_INVALID_ARG, "camera invalid (finite values, vfov in (0, 180))");
    }
    if (r.deadline_ns < 0) return bad(OCC_ERR_INVALID_ARG, "deadline_ns must be >= 0");
    const int64_t bytes = request_bytes(r);

    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return bad(OCC_ERR_INVALID_ARG, "server is shutting down");
    occ::PatternParams pp;
    occ_status st = occ::make_pattern(S->submit_ctx, &r.pattern, r.K, &pp);
    if (st == OCC_OK && r.effect == OCC_EFFECT_SHADOW) st = occ::check_light(S->submit_ctx, &r.light);
    if (st != OCC_OK) return bad(st, S->submit_ctx->last_error.c_str());
    const uint64_t rid = S->next_id++;
    const int64_t t = S->now();
    st = S->sched->submit(rid, bytes, t, r.deadline_ns > 0 ? t + r.deadline_ns : 0);
    if (st != OCC_OK) {
        std::snprintf(msg, sizeof(msg),
                      st == OCC_ERR_OOM ? "request needs %lld bytes, more than the budget"
                                        : "queue is full (%lld bytes request)",
                      (long long)bytes);
        return bad(st, msg);
    }
    Req& q = S->reqs[rid];
    q.r = r;
    if (r.pattern.kind == OCC_PAT_OFFSETS && r.pattern.n_offsets > 0) {
        q.offsets.assign(r.pattern.offsets_host, r.pattern.offsets_host + 2 * r.pattern.n_offsets);
        q.r.pattern.offsets_host = q.offsets.data();
    } else {
        q.r.pattern.offsets_host = nullptr;
    }
    q.bytes = bytes;
    q.t_submit = t;
    *id = rid;
    S->cv_work.notify_one();
    return OCC_OK;
}

OCC_EXPORT occ_status occ_server_poll(occ_server* S, occ_result* out, int32_t cap,
                                      int64_t timeout_us, int32_t* n) {
    if (!S || !out || cap < 1 || !n) return OCC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [S] { return !S->done.empty() || S->worker_exited; };
    if (timeout_us < 0)
        S->cv_done.wait(lk, ready);
    else if (timeout_us > 0)
        S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    int k = 0;
    while (k < cap && !S->done.empty()) {
        out[k++] = S->done.front();
        S->done.pop_front();
    }
    *n = k;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_server_get_stats(occ_server* S, occ_server_stats* out) {
    if (!S || !out) return OCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->sched = S->sched->stats();
    out->budget_bytes = S->cfg.budget_bytes;
    out->batches = S->batches;
    out->views_batched = S->views_batched;
    out->views_single = S->views_single;
    uint64_t v = 0;
    if (cudaMemPoolGetAttribute(S->pool, cudaMemPoolAttrReservedMemCurrent, &v) == cudaSuccess)
        out->pool_reserved_bytes = (int64_t)v;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_server_shutdown(occ_server* S, int32_t cancel_queued) {
    if (!S) return OCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> join_lk(S->join_mu);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->stop) {
            S->stop = true;
            S->cancel = cancel_queued != 0;
        }
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    return OCC_OK;
}

OCC_EXPORT occ_status occ_server_destroy(occ_server* S, int32_t cancel_queued) {
    if (!S) return OCC_ERR_INVALID_ARG;
    occ_server_shutdown(S, cancel_queued);
    release(S);
    return OCC_OK;
}
