// occ_sched.cpp -- admission scheduler of the serving loop (include/occ_serve.h):
// host-only bookkeeping, no CUDA call.  FIFO admission under a device-byte budget,
// a limit on batches in flight, a queue limit and admission deadlines.
#include <algorithm>
#include <cstring>
#include <deque>
#include <mutex>
#include <unordered_set>
#include <vector>

#include "occ_serve.h"
#include "occ_sched.h"

#define OCC_EXPORT extern "C" __attribute__((visibility("default")))

namespace occ {

Scheduler::Scheduler(const occ_sched_config& cfg)
    : cfg_(cfg), slot_bytes_(cfg.max_inflight, 0), slot_busy_(cfg.max_inflight, false) {}

bool Scheduler::valid_config(const occ_sched_config& c) {
    return c.budget_bytes > 0 && c.max_views_per_batch >= 1 && c.max_views_per_batch <= 256 &&
           c.max_inflight >= 1 && c.max_inflight <= kMaxInflight && c.max_queued >= 1;
}

occ_status Scheduler::submit(uint64_t id, int64_t bytes, int64_t now, int64_t deadline) {
    ++st_.submitted;
    if (bytes <= 0 || live_.count(id)) {
        ++st_.refused;
        return OCC_ERR_INVALID_ARG;
    }
    if (bytes > cfg_.budget_bytes) {
        ++st_.refused;
        return OCC_ERR_OOM;
    }
    if ((int64_t)q_.size() >= cfg_.max_queued) {
        ++st_.refused;
        return OCC_ERR_BUSY;
    }
    q_.push_back(Queued{id, bytes, deadline, now});
    live_.insert(id);
    st_.queued = (int64_t)q_.size();
    return OCC_OK;
}

int Scheduler::next(int64_t now, std::vector<uint64_t>* ids, int cap, std::vector<uint64_t>* expired,
                    int exp_cap, bool admit) {
    ids->clear();
    expired->clear();
    // 1. deadlines (anywhere in the queue)
    bool more_due = false;
    for (auto it = q_.begin(); it != q_.end();) {
        if (it->deadline > 0 && now > it->deadline) {
            if ((int)expired->size() >= exp_cap) {
                more_due = true;
                break;
            }
            expired->push_back(it->id);
            live_.erase(it->id);
            ++st_.expired;
            it = q_.erase(it);
        } else {
            ++it;
        }
    }
    st_.queued = (int64_t)q_.size();
    if (more_due || q_.empty() || !admit) return -1;
    // 2. a free slot, then FIFO admission within the budget
    int slot = -1;
    for (int s = 0; s < cfg_.max_inflight; ++s)
        if (!slot_busy_[s]) {
            slot = s;
            break;
        }
    if (slot < 0) return -1;
    const int limit = std::min(cap, cfg_.max_views_per_batch);
    int64_t bytes = 0;
    while (!q_.empty() && (int)ids->size() < limit &&
           st_.reserved_bytes + bytes + q_.front().bytes <= cfg_.budget_bytes) {
        bytes += q_.front().bytes;
        ids->push_back(q_.front().id);
        q_.pop_front();
    }
    st_.queued = (int64_t)q_.size();
    if (ids->empty()) return -1;
    slot_busy_[slot] = true;
    slot_bytes_[slot] = bytes;
    slot_ids_[slot] = *ids;
    st_.reserved_bytes += bytes;
    st_.peak_reserved_bytes = std::max(st_.peak_reserved_bytes, st_.reserved_bytes);
    st_.admitted += (int64_t)ids->size();
    ++st_.inflight_batches;
    return slot;
}

bool Scheduler::complete(int slot) {
    if (slot < 0 || slot >= cfg_.max_inflight || !slot_busy_[slot]) return false;
    slot_busy_[slot] = false;
    st_.reserved_bytes -= slot_bytes_[slot];
    slot_bytes_[slot] = 0;
    for (uint64_t id : slot_ids_[slot]) live_.erase(id);
    slot_ids_[slot].clear();
    --st_.inflight_batches;
    ++st_.completed_batches;
    return true;
}

int Scheduler::drain(uint64_t* ids, int cap) {
    int n = 0;
    while (!q_.empty() && n < cap) {
        ids[n++] = q_.front().id;
        live_.erase(q_.front().id);
        q_.pop_front();
    }
    st_.queued = (int64_t)q_.size();
    return n;
}

}  // namespace occ

struct occ_sched {
    std::mutex mu;
    occ::Scheduler s;
    explicit occ_sched(const occ_sched_config& c) : s(c) {}
};

OCC_EXPORT occ_status occ_sched_create(const occ_sched_config* cfg, occ_sched** out) {
    if (!cfg || !out) return OCC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!occ::Scheduler::valid_config(*cfg)) return OCC_ERR_INVALID_ARG;
    *out = new occ_sched(*cfg);
    return OCC_OK;
}

OCC_EXPORT occ_status occ_sched_destroy(occ_sched* s) {
    if (!s) return OCC_ERR_INVALID_ARG;
    delete s;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_sched_submit(occ_sched* s, uint64_t id, int64_t bytes, int64_t now_ns,
                                       int64_t deadline_ns) {
    if (!s) return OCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->s.submit(id, bytes, now_ns, deadline_ns);
}

OCC_EXPORT occ_status occ_sched_next(occ_sched* s, int64_t now_ns, uint64_t* ids, int32_t cap,
                                     int32_t* n, int32_t* slot, uint64_t* expired, int32_t exp_cap,
                                     int32_t* n_expired) {
    if (!s || !ids || cap < 1 || !n || !slot || (exp_cap > 0 && !expired) || exp_cap < 0 ||
        !n_expired)
        return OCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<uint64_t> got, exp;
    *slot = s->s.next(now_ns, &got, cap, &exp, exp_cap);
    *n = (int32_t)got.size();
    *n_expired = (int32_t)exp.size();
    if (!got.empty()) std::memcpy(ids, got.data(), got.size() * sizeof(uint64_t));
    if (!exp.empty()) std::memcpy(expired, exp.data(), exp.size() * sizeof(uint64_t));
    return OCC_OK;
}

OCC_EXPORT occ_status occ_sched_complete(occ_sched* s, int32_t slot) {
    if (!s) return OCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->s.complete(slot) ? OCC_OK : OCC_ERR_INVALID_ARG;
}

OCC_EXPORT occ_status occ_sched_drain(occ_sched* s, uint64_t* ids, int32_t cap, int32_t* n) {
    if (!s || !n || cap < 0 || (cap > 0 && !ids)) return OCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *n = s->s.drain(ids, cap);
    return OCC_OK;
}

OCC_EXPORT occ_status occ_sched_get_stats(const occ_sched* s, occ_sched_stats* out) {
    if (!s || !out) return OCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(const_cast<occ_sched*>(s)->mu);
    *out = s->s.stats();
    return OCC_OK;
}
