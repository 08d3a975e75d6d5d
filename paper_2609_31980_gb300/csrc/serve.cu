// serve.cu — the serving loop: continuous batching of fixed-radius
// self-queries arriving over time, admitted under a device-memory budget.
//
// Each slot is an independent child context with its own CUDA stream.  When
// a slot is free, the scheduler (serve_sched.h) admits the requests that have
// arrived, in order, as one batch that fits the bytes still free under the
// budget; the batch's host points are copied in, its grids built and queried
// by one frnn_query_batched call (segmented build, one persistent query
// launch per path) and its results copied back, all on the slot's stream.
// Other slots keep running meanwhile, so batches admitted while earlier ones
// are on the GPU overlap on the device.  A batch holds its bytes (inputs,
// grids, operands, outputs) until its completion event fires.  Latency is
// measured per request from its arrival to its results being in host memory.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>
#include <vector>

#include "frnn_host.h"
#include "serve_sched.h"

using namespace frnn;

namespace {

// Device bytes one request holds while in flight: its input and outputs, its
// share of the batch grid (sorted rows, maps, cell array), the tensor-core
// operands when D >= 8, and slack for alignment.
size_t request_bytes(int64_t n, int D, int K) {
    const int DP = padded_dim(D);
    const int64_t cap = cell_cap_for(n, std::min(D, kMaxAxes));
    size_t b = (size_t)n * D * 4 + (size_t)n * (4 + 8 * (size_t)K);
    b += (size_t)(n + 1 + kTcRowPad) * (4 * DP + 16 + 8) + (size_t)(cap + 1) * 4;
    if (D >= 8) b += (size_t)(n + 8 + kTcRowPad) * (4 * (size_t)((3 * D + 2 + 15) / 16 * 16) + 4);
    return b + 64 * 1024;
}

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

struct Slot {
    frnn_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* dbuf = nullptr;
    size_t dcap = 0;
    SchedBatch batch;
    bool busy = false;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" {

frnn_status frnn_serve_run(frnn_ctx* ctx, const frnn_request* reqs, int n_reqs, int D, float r,
                           int K, size_t mem_budget_bytes, int n_slots, int max_batch,
                           double* latency_ms, frnn_serve_stats* stats) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    if (n_reqs < 0 || (n_reqs > 0 && !reqs) || D < 1 || D > kMaxD || K < 1 || K > kMaxK ||
        n_slots < 1 || n_slots > 64 || max_batch < 1 || !(r > 0.f) || !std::isfinite(r))
        return FRNN_ERR_INVALID_ARG;
    for (int i = 0; i < n_reqs; ++i)
        if (reqs[i].n < 0 || (reqs[i].n > 0 && (!reqs[i].pts || !reqs[i].counts ||
                                                 !reqs[i].idx || !reqs[i].dist2)) ||
            !(reqs[i].arrival_s >= 0.0))
            return FRNN_ERR_INVALID_ARG;
    std::vector<SchedRequest> sr(n_reqs);
    for (int i = 0; i < n_reqs; ++i) sr[i] = {reqs[i].arrival_s, request_bytes(reqs[i].n, D, K)};
    const size_t budget = mem_budget_bytes ? mem_budget_bytes : (size_t)-1;
    Scheduler sched(sr, budget, n_slots, max_batch);

    std::vector<Slot> slots(n_slots);
    frnn_status status = FRNN_OK;
    for (auto& s : slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            status = FRNN_ERR_CUDA;
            break;
        }
        status = frnn_create(&s.ctx, s.stream, 0);
        if (status != FRNN_OK) break;
        // children inherit the parent's options; every batch is new, so no graph
        ctx_copy_tuning(s.ctx, ctx);
        frnn_set_option(s.ctx, FRNN_OPT_USE_GRAPH, 0);
    }

    // Warm every slot before the clock starts: its workspace for the largest
    // batch it may be given (max_batch copies of the largest request, fewer
    // when the slots' share of the budget cannot hold that many), so that no
    // allocation, and no device-wide synchronisation of cudaFree, happens
    // while other slots are running.  Larger batches still grow on demand.
    int64_t n_max = 0;
    for (int i = 0; i < n_reqs; ++i) n_max = std::max(n_max, reqs[i].n);
    if (status == FRNN_OK && n_max > 0) {
        const size_t per_req = request_bytes(n_max, D, K);
        const size_t share = budget / (size_t)n_slots;
        const int copies = (int)std::max<size_t>(
            1, std::min<size_t>((size_t)max_batch, share / std::max<size_t>(per_req, 1)));
        const size_t io = (size_t)copies * (al256((size_t)n_max * D * 4) + al256((size_t)n_max * 4) +
                                            2 * al256((size_t)n_max * K * 4));
        for (auto& s : slots) {
            status = ctx_reserve_batch(s.ctx, copies, n_max, D, K, 0);
            if (status != FRNN_OK) break;
            if (cudaMalloc(&s.dbuf, io) != cudaSuccess) {
                cudaGetLastError();
                s.dbuf = nullptr;
                status = FRNN_ERR_OUT_OF_MEMORY;
                break;
            }
            s.dcap = io;
        }
    }

    std::vector<double> finish(n_reqs, -1.0);
    const double t0 = now_s();
    std::vector<frnn_event> evs;
    std::vector<char> direct;
    auto launch = [&](Slot& s) -> frnn_status {
        const SchedBatch& b = s.batch;
        // device layout: per request input, counts, idx, dist2
        size_t need = 0;
        for (int rq : b.reqs) {
            const int64_t n = reqs[rq].n;
            need += al256((size_t)n * D * 4) + al256((size_t)n * 4) + 2 * al256((size_t)n * K * 4);
        }
        if (need > s.dcap) {
            if (s.dbuf) cudaFree(s.dbuf);   // slot idle: nothing of it in flight
            s.dbuf = nullptr;
            s.dcap = 0;
            if (cudaMalloc(&s.dbuf, need) != cudaSuccess) {
                cudaGetLastError();
                return FRNN_ERR_OUT_OF_MEMORY;
            }
            s.dcap = need;
        }
        char* p = static_cast<char*>(s.dbuf);
        evs.assign(b.reqs.size(), frnn_event{});
        direct.assign(b.reqs.size(), 0);
        for (size_t i = 0; i < b.reqs.size(); ++i) {
            const frnn_request& q = reqs[b.reqs[i]];
            const int64_t n = q.n;
            frnn_event& ev = evs[i];
            ev.n = n;
            ev.pts = reinterpret_cast<float*>(p);
            p += al256((size_t)n * D * 4);
            ev.counts = reinterpret_cast<int32_t*>(p);
            p += al256((size_t)n * 4);
            ev.idx = reinterpret_cast<int32_t*>(p);
            p += al256((size_t)n * K * 4);
            ev.dist2 = reinterpret_cast<float*>(p);
            p += al256((size_t)n * K * 4);
            // page-locked result buffers: the kernels write them directly
            void* mc = mapped_host(q.counts);
            void* mi = mapped_host(q.idx);
            void* md = mapped_host(q.dist2);
            if (mc && mi && md) {
                ev.counts = static_cast<int32_t*>(mc);
                ev.idx = static_cast<int32_t*>(mi);
                ev.dist2 = static_cast<float*>(md);
                direct[i] = 1;
            }
            if (n > 0 && cudaMemcpyAsync(const_cast<float*>(ev.pts), q.pts, (size_t)n * D * 4,
                                         cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
                return FRNN_ERR_CUDA;
        }
        frnn_status st = frnn_query_batched(s.ctx, evs.data(), (int)evs.size(), D, r, K, 0);
        if (st != FRNN_OK) return st;
        for (size_t i = 0; i < b.reqs.size(); ++i) {
            const frnn_request& q = reqs[b.reqs[i]];
            const int64_t n = q.n;
            if (n == 0 || direct[i]) continue;
            cudaMemcpyAsync(q.counts, evs[i].counts, (size_t)n * 4, cudaMemcpyDeviceToHost,
                            s.stream);
            cudaMemcpyAsync(q.idx, evs[i].idx, (size_t)n * K * 4, cudaMemcpyDeviceToHost,
                            s.stream);
            cudaMemcpyAsync(q.dist2, evs[i].dist2, (size_t)n * K * 4, cudaMemcpyDeviceToHost,
                            s.stream);
        }
        if (cudaEventRecord(s.done, s.stream) != cudaSuccess) return FRNN_ERR_CUDA;
        return FRNN_OK;
    };

    while (status == FRNN_OK && !sched.done()) {
        bool progressed = false;
        for (auto& s : slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                cudaGetLastError();
                status = FRNN_ERR_CUDA;
                break;
            }
            status = frnn_sync(s.ctx);   // device-side status of this batch
            const double t = now_s() - t0;
            for (int rq : s.batch.reqs) finish[rq] = t;
            sched.complete(s.batch);
            s.busy = false;
            progressed = true;
        }
        if (status != FRNN_OK) break;
        SchedBatch b;
        while (status == FRNN_OK && sched.next_batch(now_s() - t0, b)) {
            Slot& s = slots[b.slot];
            s.batch = b;
            s.busy = true;
            status = launch(s);
            progressed = true;
        }
        if (!progressed) {
            // nothing to complete or admit right now: wait a little (for the
            // next arrival, or a completion on the GPU)
            const double wait = sched.next_arrival() - (now_s() - t0);
            if (wait > 1e-4) std::this_thread::sleep_for(std::chrono::microseconds(20));
            else std::this_thread::yield();
        }
    }
    for (auto& s : slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
    }
    const double wall = now_s() - t0;

    // statistics
    std::vector<double> lat;
    int64_t rejected = 0;
    for (int i = 0; i < n_reqs; ++i) {
        double l = -1.0;
        if (sched.rejected(i)) {
            ++rejected;
        } else if (finish[i] >= 0.0) {
            l = (finish[i] - reqs[i].arrival_s) * 1e3;
            lat.push_back(l);
        }
        if (latency_ms) latency_ms[i] = l;
    }
    if (stats) {
        frnn_serve_stats st{};
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double p) {
            if (lat.empty()) return 0.0;
            const double pos = p * (lat.size() - 1);
            const size_t lo = (size_t)pos;
            const size_t hi = std::min(lo + 1, lat.size() - 1);
            return lat[lo] + (pos - lo) * (lat[hi] - lat[lo]);
        };
        double sum = 0.0;
        for (double l : lat) sum += l;
        double first = 1e300;
        for (int i = 0; i < n_reqs; ++i) first = std::min(first, reqs[i].arrival_s);
        double last = 0.0;
        for (double f : finish) last = std::max(last, f);
        st.wall_s = n_reqs ? last - first : 0.0;
        st.p50_ms = pct(0.5);
        st.p99_ms = pct(0.99);
        st.mean_ms = lat.empty() ? 0.0 : sum / lat.size();
        st.max_ms = lat.empty() ? 0.0 : lat.back();
        st.completed = (int64_t)lat.size();
        st.rejected = rejected;
        st.events_per_s = st.wall_s > 0 ? lat.size() / st.wall_s : 0.0;
        st.peak_inflight_bytes = (int64_t)sched.peak_bytes();
        st.peak_inflight_batches = sched.peak_batches();
        (void)wall;
        *stats = st;
    }
    for (auto& s : slots) {
        if (s.ctx) frnn_destroy(s.ctx);
        if (s.dbuf) cudaFree(s.dbuf);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (status == FRNN_OK && rejected) {
        ctx_set_error(ctx, "a request is larger than the whole memory budget");
        return FRNN_ERR_BUDGET;
    }
    return status;
}

}  // extern "C"
