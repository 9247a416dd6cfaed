// occ_sched.h -- the admission scheduler of the serving loop (host only, not thread-safe;
// the C ABI and the server guard it with their own mutex).
#pragma once
#include <cstdint>
#include <deque>
#include <unordered_set>
#include <vector>

#include "occ_serve.h"

namespace occ {

class Scheduler {
public:
    static constexpr int kMaxInflight = 16;

    explicit Scheduler(const occ_sched_config& cfg);
    static bool valid_config(const occ_sched_config& c);

    occ_status submit(uint64_t id, int64_t bytes, int64_t now, int64_t deadline);
    // Expires due requests into *expired (at most exp_cap), then admits a batch into a free
    // slot; returns the slot, or -1 when nothing was admitted.
    // admit = false: expiry only.
    int next(int64_t now, std::vector<uint64_t>* ids, int cap, std::vector<uint64_t>* expired,
             int exp_cap, bool admit = true);
    bool complete(int slot);
    int drain(uint64_t* ids, int cap);
    const occ_sched_stats& stats() const { return st_; }
    // submit time of the oldest queued request (the queue must not be empty)
    int64_t oldest_submit() const { return q_.front().t_submit; }
    const occ_sched_config& config() const { return cfg_; }

private:
    struct Queued {
        uint64_t id;
        int64_t bytes;
        int64_t deadline;
        int64_t t_submit;
    };
    occ_sched_config cfg_;
    std::deque<Queued> q_;
    std::unordered_set<uint64_t> live_;   // ids queued or running
    std::vector<int64_t> slot_bytes_;
    std::vector<bool> slot_busy_;
    std::vector<uint64_t> slot_ids_[kMaxInflight];
    occ_sched_stats st_{};
};

}  // namespace occ
