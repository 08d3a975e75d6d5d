/*
 * frnn_oracle.c — plain CPU brute-force fixed-radius nearest-neighbour oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant with the
 * CUDA library.
 *
 * What it computes (the paper's Eq. 1, Sec. 1): for each query point x_i and
 * every reference point x_j,
 *
 *     N_r(i) = { j : ||x_i - x_j||_2 <= r },
 *
 * optionally keeping at most K neighbours "in distance order" (Sec. 1, just
 * after Eq. 1).  The method is exact, so the oracle is the plain O(M*N*D)
 * definition written out (brute force is the correctness reference the paper
 * measures every variant against, Sec. 1 and Sec. 4.2).
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes):
 *   - squared distance in FP32, dimensions summed in index order 0..D-1 from
 *     s = +0, each step rounded to nearest, no fused multiply-add:
 *         d = fl(q_k - p_k);  s = fl(s + fl(d * d));
 *     (the paper flags reordered accumulation as an exactness defect, Sec. 4.2
 *     and Table 1 "Grouped loads and launch bounds");
 *   - membership is inclusive, s <= fl(r * r) (Eq. 1 uses <=);
 *   - neighbours ordered by (d^2, original index) ascending, truncated to K,
 *     count = min(degree, K); padding idx = -1, dist2 = +inf;
 *   - self-exclusion by index, not by d^2 == 0 (the paper counts "non-self"
 *     edges, Sec. 4.1).
 *
 * Build: -O2 -ffp-contract=off, never -ffast-math (FMA contraction or
 * reassociation would change the contract); IEEE gradual underflow (no
 * FTZ/DAZ), which is the default on x86-64 SSE and AArch64 Linux.
 *
 * The FP64 audit (frnn_oracle_fp64_audit) recomputes every pair's verdict as
 * sum_k ((double)q_k - (double)p_k)^2 <= (double)r * (double)r and counts the
 * pairs on which the FP32 contract and FP64 disagree.  It is informational.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs float expressions evaluated in float (FLT_EVAL_METHOD == 0)"
#endif

typedef struct {
    float d2;
    int32_t j;
} oracle_pair;

/* total order used for "distance order": (d^2, index) ascending */
static int pair_less(const oracle_pair* a, const oracle_pair* b) {
    if (a->d2 != b->d2) return a->d2 < b->d2;
    return a->j < b->j;
}

static int pair_cmp(const void* pa, const void* pb) {
    const oracle_pair* a = (const oracle_pair*)pa;
    const oracle_pair* b = (const oracle_pair*)pb;
    if (pair_less(a, b)) return -1;
    if (pair_less(b, a)) return 1;
    return 0;
}

/* The FP32 contract for one pair: index order, round to nearest, no FMA. */
static float contract_d2(const float* q, const float* p, int D) {
    float s = 0.0f;
    for (int k = 0; k < D; ++k) {
        float d = q[k] - p[k];
        float t = d * d;
        s = s + t;
    }
    return s;
}

int frnn_oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Brute-force FRNN.
 *   queries   [M, D] row-major float32
 *   query_ids [M] int64 or NULL: when given, reference j == query_ids[i] is
 *             excluded (self-query by index); NULL means distinct sets
 *   refs      [N, D] row-major float32
 *   counts    [M]    out: min(degree, K)
 *   idx       [M, K] out: neighbour indices in (d^2, index) order, -1 padded
 *   dist2     [M, K] out: the contract's d^2, +inf padded
 *   degree    [M]    out (may be NULL): untruncated degree
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int frnn_oracle_query(const float* queries, const int64_t* query_ids, int64_t M,
                      const float* refs, int64_t N, int D, float r, int K,
                      int32_t* counts, int32_t* idx, float* dist2, int64_t* degree) {
    if (M < 0 || N < 0 || D < 1 || K < 1) return -1;
    if (M > 0 && (!queries || !counts || !idx || !dist2)) return -1;
    if (N > 0 && !refs) return -1;
    const float r2 = r * r;
    int failed = 0;

#pragma omp parallel
    {
        oracle_pair* buf = (oracle_pair*)malloc(sizeof(oracle_pair) * (size_t)(N > 0 ? N : 1));
        if (!buf) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < M; ++i) {
            if (!buf) continue;
            const float* q = queries + i * (int64_t)D;
            int64_t deg = 0;
            for (int64_t j = 0; j < N; ++j) {
                if (query_ids && query_ids[i] == j) continue;
                float s = contract_d2(q, refs + j * (int64_t)D, D);
                if (s <= r2) {
                    buf[deg].d2 = s;
                    buf[deg].j = (int32_t)j;
                    ++deg;
                }
            }
            qsort(buf, (size_t)deg, sizeof(oracle_pair), pair_cmp);
            int64_t keep = deg < K ? deg : K;
            counts[i] = (int32_t)keep;
            if (degree) degree[i] = deg;
            int32_t* irow = idx + i * (int64_t)K;
            float* drow = dist2 + i * (int64_t)K;
            for (int64_t e = 0; e < K; ++e) {
                if (e < keep) {
                    irow[e] = buf[e].j;
                    drow[e] = buf[e].d2;
                } else {
                    irow[e] = -1;
                    drow[e] = INFINITY;
                }
            }
        }
        free(buf);
    }
    return failed ? -1 : 0;
}

/*
 * Untruncated degree only (same contract, no sort): the count of j with
 * d^2 <= fl(r*r), self excluded by index when query_ids is given.
 */
int frnn_oracle_degree(const float* queries, const int64_t* query_ids, int64_t M,
                       const float* refs, int64_t N, int D, float r, int64_t* degree) {
    if (M < 0 || N < 0 || D < 1 || (M > 0 && (!queries || !degree))) return -1;
    const float r2 = r * r;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < M; ++i) {
        const float* q = queries + i * (int64_t)D;
        int64_t deg = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (query_ids && query_ids[i] == j) continue;
            if (contract_d2(q, refs + j * (int64_t)D, D) <= r2) ++deg;
        }
        degree[i] = deg;
    }
    return 0;
}

/*
 * FP64 boundary audit.  For every (i, j) pair (self excluded when query_ids is
 * given) compares the FP32-contract verdict with the FP64 verdict
 *     sum_k ((double)q_k - (double)p_k)^2 <= (double)r * (double)r.
 * Writes the number of pairs accepted only by FP32 to *only32 and only by FP64
 * to *only64 and returns their sum (the crossing count), or -1 on bad input.
 */
int64_t frnn_oracle_fp64_audit(const float* queries, const int64_t* query_ids, int64_t M,
                               const float* refs, int64_t N, int D, float r,
                               int64_t* only32, int64_t* only64) {
    if (M < 0 || N < 0 || D < 1) return -1;
    const float r2 = r * r;
    const double r64 = (double)r * (double)r;
    int64_t a32 = 0, a64 = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : a32, a64)
    for (int64_t i = 0; i < M; ++i) {
        const float* q = queries + i * (int64_t)D;
        for (int64_t j = 0; j < N; ++j) {
            if (query_ids && query_ids[i] == j) continue;
            const float* p = refs + j * (int64_t)D;
            int in32 = contract_d2(q, p, D) <= r2;
            double s = 0.0;
            for (int k = 0; k < D; ++k) {
                double d = (double)q[k] - (double)p[k];
                s += d * d;
            }
            int in64 = s <= r64;
            if (in32 && !in64) ++a32;
            if (in64 && !in32) ++a64;
        }
    }
    if (only32) *only32 = a32;
    if (only64) *only64 = a64;
    return a32 + a64;
}
