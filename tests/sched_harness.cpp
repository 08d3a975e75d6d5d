// CPU harness for the serving scheduler (serve_sched.h): a fake executor
// whose batches take a modelled time; reads a scenario on stdin and prints
// per-request admission and completion times plus invariants violations.
#include <cstdio>
#include <vector>
#include <algorithm>
#include "../paper_2609_31980_gb300/csrc/serve_sched.h"

int main() {
    int n, slots, max_batch;
    double per_byte, fixed;
    unsigned long long budget;
    if (scanf("%d %llu %d %d %lf %lf", &n, &budget, &slots, &max_batch, &per_byte, &fixed) != 6) return 2;
    std::vector<frnn::SchedRequest> reqs(n);
    for (int i = 0; i < n; ++i) {
        unsigned long long b;
        if (scanf("%lf %llu", &reqs[i].arrival, &b) != 2) return 2;
        reqs[i].bytes = b;
    }
    frnn::Scheduler s(reqs, budget, slots, max_batch);
    struct Running { frnn::SchedBatch b; double end; };
    std::vector<Running> run;
    std::vector<double> admit(n, -1), finish(n, -1);
    double now = 0;
    int violations = 0, guard = 0;
    while (!s.done() && guard++ < 10000000) {
        frnn::SchedBatch b;
        while (s.next_batch(now, b)) {
            double dur = fixed;
            for (int r : b.reqs) { admit[r] = now; dur += per_byte * reqs[r].bytes; }
            run.push_back({b, now + dur});
            if (s.inflight_bytes() > budget) ++violations;
            if ((int)run.size() > slots) ++violations;
            if ((int)b.reqs.size() > max_batch) ++violations;
        }
        // advance the clock to the next event: a completion or an arrival
        double next = s.next_arrival();
        if (next <= now) next = 1e300;   // arrived, waiting for a slot or bytes: a completion comes next
        for (auto& r : run) next = std::min(next, r.end);
        if (next >= 1e299) break;
        now = std::max(now, next);
        for (size_t k = 0; k < run.size();) {
            if (run[k].end <= now) {
                for (int r : run[k].b.reqs) finish[r] = now;
                s.complete(run[k].b);
                run.erase(run.begin() + k);
            } else {
                ++k;
            }
        }
    }
    printf("violations %d peak_bytes %llu peak_batches %d done %d\n", violations,
           (unsigned long long)s.peak_bytes(), s.peak_batches(), (int)s.done());
    for (int i = 0; i < n; ++i)
        printf("%d %.9f %.9f %d\n", i, admit[i], finish[i], (int)s.rejected(i));
    return 0;
}
