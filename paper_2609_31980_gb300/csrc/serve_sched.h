// serve_sched.h — admission scheduler of the serving loop (host only, no CUDA).
//
// Continuous batching under a device-memory budget: requests arrive over
// time; whenever a slot (an independent stream of device work) is free, the
// requests that have arrived are admitted in arrival order into one batch, as
// many as fit both the batch-size limit and the bytes still free under the
// budget.  A batch holds its bytes (inputs, grids, outputs) until it
// completes; then its bytes and slot are released and the next batch can be
// admitted, possibly while other batches are still running on the device.
// A request larger than the whole budget can never run and is rejected.
//
// The executor (real CUDA streams in the library, a fake clock in the CPU
// test) calls next_batch() when it has a free slot and complete() when a
// batch finishes; the scheduler only decides what is admitted when.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <vector>

namespace frnn {

struct SchedRequest {
    double arrival;     // seconds from the start of the run
    size_t bytes;       // device bytes the request holds while in flight
};

struct SchedBatch {
    std::vector<int> reqs;   // request indices, arrival order
    size_t bytes = 0;
    int slot = -1;
};

class Scheduler {
public:
    Scheduler(const std::vector<SchedRequest>& reqs, size_t budget, int slots, int max_batch)
        : reqs_(reqs), budget_(budget), slot_busy_(slots, false),
          max_batch_(max_batch < 1 ? 1 : max_batch), state_(reqs.size(), kWaiting) {
        // arrival order (stable for equal times)
        order_.resize(reqs.size());
        for (size_t i = 0; i < reqs.size(); ++i) order_[i] = (int)i;
        for (size_t i = 1; i < order_.size(); ++i) {
            const int v = order_[i];
            size_t j = i;
            while (j > 0 && reqs_[order_[j - 1]].arrival > reqs_[v].arrival) {
                order_[j] = order_[j - 1];
                --j;
            }
            order_[j] = v;
        }
    }

    // Admit a batch at time `now` if a slot is free and the request at the
    // head of the queue has arrived and fits.  Requests that can never fit
    // are rejected (state kRejected) as they reach the head.
    bool next_batch(double now, SchedBatch& out) {
        int slot = -1;
        for (size_t s = 0; s < slot_busy_.size(); ++s)
            if (!slot_busy_[s]) {
                slot = (int)s;
                break;
            }
        if (slot < 0) return false;
        out = SchedBatch();
        while (head_ < order_.size()) {
            const int r = order_[head_];
            if (reqs_[r].arrival > now) break;
            if (reqs_[r].bytes > budget_) {
                state_[r] = kRejected;
                ++head_;
                ++finished_;
                continue;
            }
            if ((int)out.reqs.size() >= max_batch_) break;
            if (inflight_ + out.bytes + reqs_[r].bytes > budget_) break;   // head-of-line: FIFO
            out.reqs.push_back(r);
            out.bytes += reqs_[r].bytes;
            state_[r] = kRunning;
            ++head_;
        }
        if (out.reqs.empty()) return false;
        out.slot = slot;
        slot_busy_[slot] = true;
        inflight_ += out.bytes;
        if (inflight_ > peak_bytes_) peak_bytes_ = inflight_;
        ++inflight_batches_;
        if (inflight_batches_ > peak_batches_) peak_batches_ = inflight_batches_;
        return true;
    }

    void complete(const SchedBatch& b) {
        slot_busy_[b.slot] = false;
        inflight_ -= b.bytes;
        --inflight_batches_;
        for (int r : b.reqs) {
            state_[r] = kDone;
            ++finished_;
        }
    }

    bool done() const { return finished_ == reqs_.size(); }
    // arrival time of the next request not yet admitted (or a huge value)
    double next_arrival() const {
        return head_ < order_.size() ? reqs_[order_[head_]].arrival : 1e300;
    }
    bool rejected(int r) const { return state_[r] == kRejected; }
    size_t inflight_bytes() const { return inflight_; }
    size_t peak_bytes() const { return peak_bytes_; }
    int peak_batches() const { return peak_batches_; }

private:
    enum State { kWaiting, kRunning, kDone, kRejected };
    std::vector<SchedRequest> reqs_;
    size_t budget_;
    std::vector<bool> slot_busy_;
    int max_batch_;
    std::vector<int> order_;
    std::vector<State> state_;
    size_t head_ = 0;
    size_t finished_ = 0;
    size_t inflight_ = 0;
    size_t peak_bytes_ = 0;
    int inflight_batches_ = 0;
    int peak_batches_ = 0;
};

}  // namespace frnn
