// query.cu — grid-path fixed-radius query: per-warp scan of the neighbouring
// cells with candidate tiles staged in shared memory by bulk copies, the exact
// float32 distance contract, and warp-level top-K.
//
// Method (Eq. 1, Sec. 1): for each query, every reference in the cells within
// +-m cells along each gridded axis is a candidate (complete by the grid's
// roundoff-safe construction, build.cu); each candidate's squared distance is
// computed under the fixed float32 contract and kept if <= fl(r*r).
//
// Organisation on the GPU (differs from the paper's thread-per-query kernel,
// whose profile showed dependent-load latency and divergence, Sec. 4.2):
//   * a persistent grid; each warp takes chunks of kChunkQ consecutive
//     cell-sorted query slots from an atomic counter (no task list: the chunk
//     number alone locates the slots).  Runs of queries of a chunk whose
//     cells are equal or follow each other along the fastest axis of one row
//     form a group; a group's candidates are the points of its neighbour
//     rows (every gridded coordinate but the fastest within +-m), each
//     restricted to the cells from m before the group's first cell to m
//     after its last along the fastest axis: one contiguous slot range per
//     neighbour row, a superset of each query's own +-m neighbourhood;
//   * the warp enumerates the neighbour rows of its groups 32 at a time
//     (lanes), keeps the non-empty ranges in a compact list and concatenates
//     them into one candidate stream, group after group;
//   * the stream is cut into tiles of TILE candidates; every range part of a
//     tile is copied from HBM/L2 into the warp's shared-memory ring with one
//     cp.async.bulk (cell-sorted points are plain rows, so a slot range is one
//     contiguous block), completion tracked by one mbarrier per buffer, the
//     next tile in flight while the current one is evaluated;
//   * evaluation puts candidates on lanes: each lane takes one candidate of
//     the tile and computes the contract's squared distance to every query of
//     that candidate's group (__fsub_rn / __fmul_rn / __fadd_rn in index
//     order, never contracted), so lanes stay busy however few queries share
//     a cell.  Accepted pairs (d2, slot) are appended to the query's list in
//     shared memory (at most kListCap; a longer list sends the row to the
//     exact selection kernel);
//   * for each query the warp loads the list (entry e on lane e), resolves the
//     original indices (the deferred lookup, Table 3), sorts the keys (d2 bits
//     << 32 | original index) with a bitonic network across the lanes, only as
//     wide as the row, and writes the first K (count = min(degree, K))
//     coalesced, with the padding.  Lists longer than kListCap go to an exact
//     selection kernel, keeping results exact for dense inputs (the paper's
//     Sec. 5 caveat on heap-free top-K).
#include <algorithm>
#include <climits>
#include <cmath>

#include "frnn_host.h"

namespace frnn {

constexpr int kQueryWarps = 4;
constexpr uint32_t kFull = 0xffffffffu;
constexpr int kListCap = 32;      // accepted entries a query keeps in the kernel (one per lane)
constexpr int kListStr = 33;      // list row stride (entries): conflict-free both ways
constexpr int kRangeCap = 128;    // compact candidate ranges of one batch of groups
constexpr int kNbrRounds = kMaxNbrRows / 32;
static_assert(kListCap <= kCsrStageW, "a staged compact row holds a whole kernel row");
static_assert(kRangeCap >= kMaxNbrRows, "one group's ranges always fit a batch");
static_assert(kChunkQ <= 16, "group search over at most 16 groups");

// Candidate staging.  kStageLoads: each lane loads its candidate's row from
// global memory (the cell-sorted rows of an event stay L2-resident), the next
// round's rows in flight while the current round is evaluated.  kStageBulk:
// the stream is cut into tiles that cp.async.bulk copies into a two-buffer
// shared-memory ring (one copy per range part, completion on an mbarrier).
constexpr int kStageLoads = 0;
constexpr int kStageBulk = 1;

template <int D, int STAGE>
struct QCfg {
    static constexpr int DP = padded_dim(D);
    // candidates per tile and ring buffers of the bulk-copy staging
    static constexpr int TILE = 64;
    static constexpr int NB = 2;
    // CTAs per SM (the scan is latency-bound and wants resident warps): as
    // many as the per-warp shared memory and the registers allow
    static constexpr int MINB = STAGE == kStageBulk
                                    ? (DP <= 4 ? 6 : (DP <= 8 ? 5 : (DP <= 12 ? 4 : 3)))
                                    : (DP <= 8 ? 6 : (DP <= 12 ? 4 : 3));
    // sort two short query rows at once, one per half-warp (rows of at most
    // 16 entries: the 500k x 12 event's clustered queries have about 12)
    static constexpr bool PAIR_ROWS = D >= 10;
};

// Per-warp shared memory.  Every bulk-copy destination (the ring) starts on
// a 128-byte boundary and holds whole rows of DP floats (16-byte multiples).
struct WarpSmem {
    float* ring;      // [NB][TILE][DP] candidate coordinates (bulk staging)
    int32_t* tslot;   // [NB][TILE] candidate slots (bulk staging)
    float* Q;         // [kChunkQ][DP] the chunk's query coordinates
    float* Ld;        // [kChunkQ][kListStr] accepted squared distances
    int32_t* Li;      // [kChunkQ][kListStr] accepted slots, then original indices
    uint64_t* bars;   // [NB] (bulk staging)
    int32_t* rlo;     // [kRangeCap] first slot of each compact range
    int32_t* rpre;    // [kRangeCap + 1] stream position of each range; sentinel = length
    int32_t* cnt;     // [kChunkQ] accepted entries per query
    int32_t* tdelta;  // [kNbrRounds][32] neighbour-row table: offsets (table_in_smem only)
    uint32_t* tedge;  // [kNbrRounds][32] neighbour-row table: edge codes (table_in_smem only)
};

constexpr size_t kSmemPerSm = 228 * 1024;      // shared memory of one SM
constexpr size_t kSmemPerCtaReserved = 1024;   // taken by the system from each resident CTA
constexpr size_t kNbrTableBytes = 2 * (size_t)kNbrRounds * 32 * 4;

template <int D, int STAGE>
__host__ __device__ constexpr size_t warp_smem_core_bytes() {
    using C = QCfg<D, STAGE>;
    constexpr size_t ring = STAGE == kStageBulk ? (size_t)C::NB * C::TILE * (C::DP + 1) * 4 + C::NB * 8 : 0;
    return ring + (size_t)kChunkQ * C::DP * 4 + 2 * (size_t)kChunkQ * kListStr * 4 + (size_t)kRangeCap * 4 +
           (size_t)(kRangeCap + 1) * 4 + (size_t)kChunkQ * 4;
}

// The neighbour-row table lives in shared memory (which frees eight
// registers a lane for the scan) wherever that still lets MINB CTAs reside
// on an SM; otherwise in registers.
template <int D, int STAGE>
__host__ __device__ constexpr bool table_in_smem() {
    return (kQueryWarps * ((warp_smem_core_bytes<D, STAGE>() + kNbrTableBytes + 127) / 128 * 128) +
            kSmemPerCtaReserved) * QCfg<D, STAGE>::MINB <= kSmemPerSm;
}

template <int D, int STAGE>
__host__ __device__ constexpr size_t warp_smem_bytes() {
    return (warp_smem_core_bytes<D, STAGE>() + (table_in_smem<D, STAGE>() ? kNbrTableBytes : 0) + 127) /
           128 * 128;
}

// The table's two words for row l = 32 rr + lane, in registers or in the
// warp's shared memory (row-major by rr, one word per lane: conflict-free).
template <bool SMEM>
struct NbrTable {
    int32_t d[kNbrRounds];
    uint32_t e[kNbrRounds];
    __device__ __forceinline__ NbrTable(const WarpSmem&, int) {}
    __device__ __forceinline__ int32_t& delta(int rr) { return d[rr]; }
    __device__ __forceinline__ uint32_t& edge(int rr) { return e[rr]; }
};
template <>
struct NbrTable<true> {
    int32_t* d;
    uint32_t* e;
    __device__ __forceinline__ NbrTable(const WarpSmem& w, int lane) : d(w.tdelta + lane), e(w.tedge + lane) {}
    __device__ __forceinline__ int32_t& delta(int rr) { return d[rr * 32]; }
    __device__ __forceinline__ uint32_t& edge(int rr) { return e[rr * 32]; }
};

template <int D, int STAGE>
__device__ __forceinline__ WarpSmem carve_warp(unsigned char* base) {
    using C = QCfg<D, STAGE>;
    constexpr int NBUF = STAGE == kStageBulk ? C::NB : 0;
    WarpSmem w;
    w.ring = reinterpret_cast<float*>(base);
    w.tslot = reinterpret_cast<int32_t*>(w.ring + NBUF * C::TILE * C::DP);
    w.Q = reinterpret_cast<float*>(w.tslot + NBUF * C::TILE);
    w.Ld = w.Q + kChunkQ * C::DP;
    w.Li = reinterpret_cast<int32_t*>(w.Ld + kChunkQ * kListStr);
    w.bars = reinterpret_cast<uint64_t*>(w.Li + kChunkQ * kListStr);
    w.rlo = reinterpret_cast<int32_t*>(w.bars + NBUF);
    w.rpre = w.rlo + kRangeCap;
    w.cnt = w.rpre + kRangeCap + 1;
    w.tdelta = w.cnt + kChunkQ;   // past the end of the warp's area unless table_in_smem
    w.tedge = reinterpret_cast<uint32_t*>(w.tdelta + kNbrRounds * 32);
    return w;
}

__device__ __forceinline__ uint64_t make_key(float d2, int32_t j) {
    return ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)j;
}

// Event of a chunk: the last event whose first chunk is <= c.
__device__ __forceinline__ int chunk_event(const EventHdr* qev, int E, int c) {
    int lo = 0, hi = E - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (qev[mid].qchunk0 <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Copy tile t of the batch's candidate stream into ring buffer b: every range
// part inside [T0, T1) with one bulk copy (issued by the lane holding the
// range), the slots of the copied candidates into tslot, completion on the
// buffer's mbarrier.  cur: first range that may overlap the tile (advanced).
template <int D, int STAGE>
__device__ __forceinline__ void issue_tile(const WarpSmem& w, int t, int b, int U, int nr,
                                           int& cur, const float* rpts, int lane) {
    using C = QCfg<D, STAGE>;
    constexpr int DP = C::DP, T = C::TILE;
    const int T0 = t * T;
    const int T1 = min(T0 + T, U);
    if (lane == 0) mbar_arrive_expect_tx(&w.bars[b], (uint32_t)(T1 - T0) * DP * sizeof(float));
    __syncwarp();
    fence_proxy_async_smem();   // the buffer's previous contents were read generically
    for (int i = cur + lane; i < nr; i += 32) {
        const int ps = w.rpre[i];
        if (ps >= T1) break;
        const int pe = w.rpre[i + 1];
        const int s = max(ps, T0), e = min(pe, T1);
        if (e > s) {
            const int lo = w.rlo[i] + (s - ps);
            bulk_g2s(w.ring + ((size_t)b * T + (s - T0)) * DP, rpts + (int64_t)lo * DP,
                     (uint32_t)(e - s) * DP * sizeof(float), &w.bars[b]);
            int32_t* ts = w.tslot + b * T + (s - T0);
            for (int j = 0; j < e - s; ++j) ts[j] = lo + j;
        }
    }
    // the first range still reaching past this tile
    while (cur < nr && w.rpre[cur + 1] <= T1) ++cur;
}

template <int D, int STAGE>
__global__ void __launch_bounds__(kQueryWarps * 32, QCfg<D, STAGE>::MINB) k_grid_query(QueryArgs a) {
    pdl_trigger();
    pdl_wait();
    using C = QCfg<D, STAGE>;
    constexpr int DP = C::DP;
    constexpr int T = C::TILE;
    constexpr int NB = C::NB;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpSmem w = carve_warp<D, STAGE>(smem + (size_t)warp * warp_smem_bytes<D, STAGE>());
    if constexpr (STAGE == kStageBulk) {
        if (lane == 0)
            for (int b = 0; b < NB; ++b) mbar_init(&w.bars[b], 1);
        fence_mbar_init();
        __syncwarp();
    }
    uint32_t phase = 0;   // bit b: parity to wait for on buffer b (bulk staging)
    const unsigned lt_mask = (1u << lane) - 1u;

    const float r2 = a.r2;
    const int K = a.K;
    // neighbour-row table of the current event, for row l = 32 rr + lane:
    // tab.delta(rr) = its linear offset from the group's row; tab.edge(rr) =
    // for m = 1 the axes whose offset is -1 (bits 0-3) and +1 (bits 8-11), for
    // larger m the offsets + m (3 bits per axis); bit 31: l is beyond the rows
    int tab_e = -1;
    NbrTable<table_in_smem<D, STAGE>()> tab(w, lane);

    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(a.task_counter, 1);
        c = __shfl_sync(kFull, c, 0);
        if (c >= a.nchunks) break;
        const int e = a.nev > 1 ? chunk_event(a.qev, a.nev, c) : 0;
        const EventHdr& hq = a.qev[e];
        const EventHdr& h = a.ev[e];
        if (a.path_filter >= 0 && h.path != a.path_filter) continue;   // another launch's event
        int32_t* counts = a.counts ? a.counts : h.counts;
        int32_t* oidx = a.counts ? a.idx : h.idx;
        float* od2 = a.counts ? a.dist2 : h.dist2;

        const int64_t q_off = hq.pt_off, q_n = hq.n;
        const int s0 = (int)(q_off + (int64_t)(c - hq.qchunk0) * kChunkQ);
        const int nqc = (int)min((int64_t)kChunkQ, q_off + q_n - (int64_t)s0);
        const bool act = lane < nqc;
        const int qs = s0 + lane;
        const int qorig = act ? a.qperm[qs] : 0;
        if (!h.valid) {
            // grid built from non-finite input: empty rows (frnn_sync reports it)
            for (int ql = 0; ql < nqc && !a.csr; ++ql) {
                const int qo = __shfl_sync(kFull, qorig, ql);
                for (int e2 = lane; e2 < K; e2 += 32) {
                    oidx[(int64_t)qo * K + e2] = -1;
                    od2[(int64_t)qo * K + e2] = INFINITY;
                }
            }
            if (act) counts[qorig] = 0;
            if (act && a.degree) a.degree[qorig] = 0;
            continue;
        }
        // the chunk's query rows into shared memory; per-query counters
        {
            const float4* src = reinterpret_cast<const float4*>(a.qpts + (int64_t)s0 * DP);
            float4* dst = reinterpret_cast<float4*>(w.Q);
            for (int i = lane; i < nqc * (DP / 4); i += 32) dst[i] = src[i];
            if (lane < kChunkQ) w.cnt[lane] = 0;
        }
        const int qc = act ? a.qcell[qs] : -1;
        const int prev = __shfl_up_sync(kFull, qc, 1);
        // the grid's parameters in registers (the loops below store to shared
        // memory through generic pointers, which would otherwise force the
        // header to be read again)
        const int naxes = h.naxes, m = h.m;
        int dims[kMaxAxes];
#pragma unroll
        for (int ax = 0; ax < kMaxAxes; ++ax) dims[ax] = h.dims[ax];
        const int dims0 = dims[0];
        const int64_t cell_off = h.cell_off;
        // this lane's cell coordinates (c0 along the fastest axis, then the row's)
        int cc[kMaxAxes];
        {
            int v = act ? qc : 0;
            cc[0] = v % dims0;
            v /= dims0;
#pragma unroll
            for (int ax = 1; ax < kMaxAxes; ++ax) {
                cc[ax] = 0;
                if (ax < naxes) {
                    cc[ax] = v % dims[ax];
                    v /= dims[ax];
                }
            }
        }
        int nrows = 1;
        for (int ax = 1; ax < naxes; ++ax) nrows *= 2 * m + 1;
        // groups: runs of queries (slots are cell-sorted) whose cells are equal
        // or follow each other along the fastest axis of one row; a group scans
        // the union of its cells' neighbourhoods, one range per neighbour row
        const bool head = act && (lane == 0 || !(qc == prev || (qc == prev + 1 && cc[0] != 0)));
        const unsigned gmask = __ballot_sync(kFull, head);
        const int ng = __popc(gmask);
        // lane g < ng: first query of group g; lanes >= ng: nqc
        int gq = nqc;
        {
            unsigned mm = gmask;
            for (int g = 0; g < ng; ++g) {
                if (lane == g) gq = __ffs(mm) - 1;
                mm &= mm - 1u;
            }
        }
        int rstride[kMaxAxes];
        rstride[0] = 0;
        rstride[1] = 1;
#pragma unroll
        for (int ax = 2; ax < kMaxAxes; ++ax) rstride[ax] = rstride[ax - 1] * dims[ax - 1];
        if (e != tab_e) {
            tab_e = e;
            const int side = 2 * m + 1;
#pragma unroll
            for (int rr = 0; rr < kNbrRounds; ++rr) {
                const int l = rr * 32 + lane;
                int ll = l, dl = 0;
                uint32_t dg = 0, lowm = 0, highm = 0;
                for (int ax = 1; ax < naxes; ++ax) {
                    const int d = ll % side;
                    ll /= side;
                    dg |= (uint32_t)d << (3 * (ax - 1));
                    dl += (d - m) * rstride[ax];
                    if (d < m) lowm |= 1u << (ax - 1);
                    if (d > m) highm |= 1u << (ax - 1);
                }
                tab.delta(rr) = dl;
                tab.edge(rr) = (m == 1 ? (lowm | (highm << 8)) : dg) | (l >= nrows ? (1u << 31) : 0u);
            }
        }

        // Row ranges of group g (lane l of round rr: neighbour row 32 rr + l):
        // every round's two cell-start loads are issued together, and the next
        // group's are issued before the current group is compacted.
        int nlo[kNbrRounds], nhi[kNbrRounds];
        auto fetch = [&](int g) {
            const int hl = __shfl_sync(kFull, gq, g);
            const int hn = __shfl_sync(kFull, gq, g + 1);   // first query of the next group, or nqc
            int gc[kMaxAxes];
#pragma unroll
            for (int ax = 0; ax < kMaxAxes; ++ax) gc[ax] = __shfl_sync(kFull, cc[ax], hl);
            const int xl = __shfl_sync(kFull, cc[0], hn - 1);   // the group's last cell on the row
            const int x0 = max(gc[0] - m, 0), x1 = min(xl + m, dims0 - 1);
            // the group's row and, for m = 1, the axes on which it touches the
            // grid's low (bits 0-3) or high (bits 8-11) edge
            int grow = 0;
            uint32_t gedge = 1u << 31;
#pragma unroll
            for (int ax = 1; ax < kMaxAxes; ++ax) {
                if (ax < naxes) {
                    grow += gc[ax] * rstride[ax];
                    if (gc[ax] == 0) gedge |= 1u << (ax - 1);
                    if (gc[ax] == dims[ax] - 1) gedge |= 1u << (ax + 7);
                }
            }
#pragma unroll
            for (int rr = 0; rr < kNbrRounds; ++rr) {
                nlo[rr] = 0;
                nhi[rr] = 0;
                if (rr * 32 < nrows) {
                    bool ok;
                    if (m == 1) {
                        ok = (tab.edge(rr) & gedge) == 0;   // in range on every axis, row exists
                    } else {
                        ok = !(tab.edge(rr) >> 31);
#pragma unroll
                        for (int ax = 1; ax < kMaxAxes; ++ax) {
                            if (ax < naxes) {
                                const int v = gc[ax] + (int)((tab.edge(rr) >> (3 * (ax - 1))) & 7u) - m;
                                ok = ok && (unsigned)v < (unsigned)dims[ax];
                            }
                        }
                    }
                    if (ok) {
                        const int64_t base = cell_off + (int64_t)(grow + tab.delta(rr)) * dims0;
                        nlo[rr] = __ldg(a.cstart + base + x0);
                        nhi[rr] = __ldg(a.cstart + base + x1 + 1);
                    }
                }
            }
        };

        // batches of groups whose compact ranges fit kRangeCap
        bool timed_out = false;
        int g0 = 0, pf = -1;   // pf: group whose ranges nlo/nhi hold
        while (g0 < ng && !timed_out) {
            int nr = 0, g = g0;
            int gr = 0;   // lane j: first compact range of batch group g0 + j
            if (pf != g0) {
                fetch(g0);
                pf = g0;
            }
            for (; g < ng; ++g) {
                int clo[kNbrRounds], chi[kNbrRounds];
#pragma unroll
                for (int rr = 0; rr < kNbrRounds; ++rr) {
                    clo[rr] = nlo[rr];
                    chi[rr] = nhi[rr];
                }
                if (g + 1 < ng) {
                    fetch(g + 1);
                    pf = g + 1;
                }
                const int nr0 = nr;
#pragma unroll
                for (int rr = 0; rr < kNbrRounds; ++rr) {
                    if (rr * 32 >= nrows) break;
                    const int lo = clo[rr];
                    const int n = chi[rr] - lo;
                    const unsigned bal = __ballot_sync(kFull, n > 0);
                    const int pos = nr + __popc(bal & lt_mask);
                    if (n > 0 && pos < kRangeCap) {
                        w.rlo[pos] = lo;
                        w.rpre[pos] = n;   // a count until the batch's scan
                    }
                    nr += __popc(bal);
                }
                if (nr > kRangeCap) {   // group g opens the next batch
                    nr = nr0;
                    break;
                }
                if (lane == g - g0) gr = nr0;
            }
            const int gend = g;
            // lane j <= gend - g0: first query of batch group j (the end for j = gend - g0)
            const int gqb = __shfl_sync(kFull, gq, min(g0 + lane, 31));
            // one exclusive scan turns the ranges' counts into stream positions
            __syncwarp();
            int U = 0;
            for (int b0 = 0; b0 < nr; b0 += 32) {
                const int i = b0 + lane;
                const int v = i < nr ? w.rpre[i] : 0;
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
                if (i < nr) w.rpre[i] = U + incl - v;
                U += __shfl_sync(kFull, incl, 31);
            }
            if (lane == 0) w.rpre[nr] = U;
            __syncwarp();
            // lane j: stream start of batch group g0 + j (INT_MAX beyond the batch)
            const int gsb = lane < gend - g0 ? w.rpre[gr] : INT_MAX;

            // one round: candidate u = k0 + lane of the stream (coordinates cv,
            // slot) against every query of its group, exact contract
            auto eval_round = [&](int u, bool valid, const float (&cv)[DP], int slot) {
                // group of the candidate: last batch group starting at or before u
                int j = 0;
#pragma unroll
                for (int st = 8; st > 0; st >>= 1) {
                    const int v = __shfl_sync(kFull, gsb, j + st);
                    if (v <= u) j += st;
                }
                const int qa = __shfl_sync(kFull, gqb, j);
                const int qe = __shfl_sync(kFull, gqb, j + 1);
                const int nq = valid ? qe - qa : 0;
                const int mx = __reduce_max_sync(kFull, (unsigned)nq);
                for (int jq = 0; jq < mx; ++jq) {
                    const bool on = jq < nq;
                    const int q = on ? qa + jq : 0;
                    const float4* qp4 = reinterpret_cast<const float4*>(w.Q + q * DP);
                    float qv[DP];
#pragma unroll
                    for (int k4 = 0; k4 < DP / 4; ++k4) {
                        const float4 v = qp4[k4];
                        qv[4 * k4] = v.x;
                        qv[4 * k4 + 1] = v.y;
                        qv[4 * k4 + 2] = v.z;
                        qv[4 * k4 + 3] = v.w;
                    }
                    // the whole contract for every candidate: a warp vote after
                    // the first dimensions (exact early rejection) was measured
                    // slower on grids of three, four and five axes alike, since a
                    // round of 32 candidates usually holds a neighbour of the query
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float d = __fsub_rn(qv[k], cv[k]);
                        s = __fadd_rn(s, __fmul_rn(d, d));
                    }
                    const bool acc = on && s <= r2 && !(a.self && slot == s0 + q);
                    if (acc) {
                        const int p = atomicAdd(&w.cnt[q], 1);
                        if (p < kListCap) {
                            w.Ld[q * kListStr + p] = s;
                            w.Li[q * kListStr + p] = slot;
                        }
                    }
                }
            };

            if constexpr (STAGE == kStageLoads) {
                // candidate u: its range by binary search over the stream
                // positions, its row loaded from global memory
                auto load_cand = [&](int u, int& slot, float (&cv)[DP]) {
                    slot = -1;
#pragma unroll
                    for (int k = 0; k < DP; ++k) cv[k] = 0.f;
                    if (u < U) {
                        int i = 0;
#pragma unroll
                        for (int st = kRangeCap / 2; st > 0; st >>= 1)
                            if (i + st < nr && w.rpre[i + st] <= u) i += st;
                        slot = w.rlo[i] + (u - w.rpre[i]);
                        const float4* p = reinterpret_cast<const float4*>(a.rpts + (int64_t)slot * DP);
#pragma unroll
                        for (int k4 = 0; k4 < DP / 4; ++k4) {
                            const float4 v = __ldg(p + k4);
                            cv[4 * k4] = v.x;
                            cv[4 * k4 + 1] = v.y;
                            cv[4 * k4 + 2] = v.z;
                            cv[4 * k4 + 3] = v.w;
                        }
                    }
                };
                int slot;
                float cv[DP];
                load_cand(lane, slot, cv);
#pragma unroll 1
                for (int k0 = 0; k0 < U; k0 += 32) {
                    int slot_n;
                    float cvn[DP];
                    load_cand(k0 + 32 + lane, slot_n, cvn);   // next round in flight
                    eval_round(k0 + lane, k0 + lane < U, cv, slot);
                    slot = slot_n;
#pragma unroll
                    for (int k = 0; k < DP; ++k) cv[k] = cvn[k];
                }
            } else {
                const int ntiles = (U + T - 1) / T;
                int cur = 0;
                const int pre = min(NB, ntiles);
                for (int tt = 0; tt < pre; ++tt) issue_tile<D, STAGE>(w, tt, tt, U, nr, cur, a.rpts, lane);
                __syncwarp();   // slots written by the issuing lanes, before any lane reads them
                int tt = 0;
                for (; tt < ntiles; ++tt) {
                    const int b = tt % NB;
                    // warp-uniform verdict: every lane takes the timeout path if one does
                    if (!__all_sync(kFull, mbar_wait_bounded(&w.bars[b], (phase >> b) & 1u))) {
                        timed_out = true;
                        break;
                    }
                    phase ^= 1u << b;
                    const int T0 = tt * T;
                    const int len = min(T, U - T0);
                    const float* tile = w.ring + (size_t)b * T * DP;
                    const int32_t* tsl = w.tslot + b * T;
#pragma unroll 1
                    for (int k0 = 0; k0 < len; k0 += 32) {
                        const int ul = k0 + lane;
                        const bool valid = ul < len;
                        float cv[DP];
                        const float4* cp = reinterpret_cast<const float4*>(tile + (size_t)(valid ? ul : 0) * DP);
#pragma unroll
                        for (int k4 = 0; k4 < DP / 4; ++k4) {
                            const float4 v = cp[k4];
                            cv[4 * k4] = v.x;
                            cv[4 * k4 + 1] = v.y;
                            cv[4 * k4 + 2] = v.z;
                            cv[4 * k4 + 3] = v.w;
                        }
                        eval_round(T0 + ul, valid, cv, valid ? tsl[ul] : -1);
                    }
                    __syncwarp();
                    if (tt + NB < ntiles) issue_tile<D, STAGE>(w, tt + NB, b, U, nr, cur, a.rpts, lane);
                }
                if (timed_out) {
                    // record, wait (bounded) for the copies still in flight, stop this warp
                    if (lane == 0) atomicOr(a.status, kStatusTimeout);
                    const int issued = min(ntiles, tt + NB);
                    for (int t2 = tt; t2 < issued; ++t2) {
                        const int b2 = t2 % NB;
                        mbar_wait_bounded(&w.bars[b2], (phase >> b2) & 1u);
                        phase ^= 1u << b2;
                    }
                    return;
                }
            }
            __syncwarp();   // the batch's ranges are rewritten by the next batch
            g0 = gend;
        }
        __syncwarp();

        // per query: counts, degree, rows for the selection kernel
        const int kept = act ? w.cnt[lane] : 0;
        const bool spill = act && kept > kListCap;
        if (act && !spill) counts[qorig] = min(kept, K);
        if (spill && a.csr) counts[qorig] = kCsrSpill;   // counted by the selection kernel
        if (act && !spill && a.degree) a.degree[qorig] = kept;
        if (spill) {
            const int pos = atomicAdd(a.ovf_count, 1);
            if (pos < a.ovf_cap) {
                a.ovf[pos].qslot = qs;
                a.ovf[pos].ev = e;
            } else {
                atomicOr(a.status, kStatusCapacity);
            }
        }
        const unsigned spill_mask = __ballot_sync(kFull, spill);
        // original indices of the kept entries (entry lane of each query),
        // all loads issued before the first store
        {
            int orig[kChunkQ];
#pragma unroll
            for (int q = 0; q < kChunkQ; ++q) {
                const int cq = __shfl_sync(kFull, kept, q);
                orig[q] = 0;
                if (q < nqc && !((spill_mask >> q) & 1u) && lane < cq)
                    orig[q] = a.rperm[w.Li[q * kListStr + lane]];
            }
#pragma unroll
            for (int q = 0; q < kChunkQ; ++q) {
                const int cq = __shfl_sync(kFull, kept, q);
                if (q < nqc && !((spill_mask >> q) & 1u) && lane < cq) w.Li[q * kListStr + lane] = orig[q];
            }
        }
        __syncwarp();
        // one query row at a time (for D >= 10 two short rows at a time, one
        // per half-warp): lane l takes entry l of the query's list, the warp
        // sorts the keys (unused lanes hold the largest key) with a bitonic
        // network across lanes, and lane l writes position l of the row
        // (coalesced), then the padding
        const int rstride_out = a.csr ? kCsrStageW : K;
        if constexpr (!C::PAIR_ROWS) {
            // two rows at a time, each in its own key: the two networks'
            // shuffle-compare chains are independent, so their latencies
            // overlap (a full-width network sorts any row, so the pair takes
            // the wider row's width)
            auto write_row = [&](int ql, int n, uint64_t key) {
                const int cK = min(n, K);
                const int qo = __shfl_sync(kFull, qorig, ql);
                int32_t* irow = oidx + (int64_t)qo * rstride_out;
                float* drow = od2 + (int64_t)qo * rstride_out;
                if (lane < cK) {
                    irow[lane] = (int32_t)(uint32_t)key;
                    drow[lane] = __uint_as_float((uint32_t)(key >> 32));
                } else if (!a.csr && lane < K) {
                    irow[lane] = -1;
                    drow[lane] = INFINITY;
                }
                for (int e2 = 32 + lane; e2 < K && !a.csr; e2 += 32) {
                    irow[e2] = -1;
                    drow[e2] = INFINITY;
                }
            };
            const unsigned rows_left = ((nqc >= 32 ? 0xffffffffu : ((1u << nqc) - 1u))) & ~spill_mask;
            unsigned todo = rows_left;
            while (todo) {
                const int qa = __ffs(todo) - 1;
                todo &= todo - 1u;
                const int qb = todo ? __ffs(todo) - 1 : -1;
                if (todo) todo &= todo - 1u;
                const int na = __shfl_sync(kFull, kept, qa);
                const int nb = __shfl_sync(kFull, kept, qb < 0 ? qa : qb);
                uint64_t ka = ~0ull, kb = ~0ull;
                if (lane < na) ka = make_key(w.Ld[qa * kListStr + lane], w.Li[qa * kListStr + lane]);
                if (qb >= 0 && lane < nb) kb = make_key(w.Ld[qb * kListStr + lane], w.Li[qb * kListStr + lane]);
                const int width = qb >= 0 ? max(na, nb) : na;
#pragma unroll
                for (int k2 = 2; k2 <= 32; k2 <<= 1) {
                    if ((k2 >> 1) >= width) break;
#pragma unroll
                    for (int jj = k2 >> 1; jj > 0; jj >>= 1) {
                        const uint64_t oa = __shfl_xor_sync(kFull, ka, jj);
                        const uint64_t ob = __shfl_xor_sync(kFull, kb, jj);
                        const bool take_min = ((lane & jj) == 0) == ((lane & k2) == 0);
                        ka = (take_min == (oa < ka)) ? oa : ka;
                        kb = (take_min == (ob < kb)) ? ob : kb;
                    }
                }
                write_row(qa, na, ka);
                if (qb >= 0) write_row(qb, nb, kb);
            }
        } else {
            // two rows at a time, one per half-warp, when both hold at most
            // 16 entries (the network then stays within each half and both
            // halves end ascending); otherwise one row per warp as above
            for (int ql = 0; ql < nqc;) {
                if ((spill_mask >> ql) & 1u) {
                    ++ql;
                    continue;
                }
                const int ql1 = ql + 1;
                const int n0 = __shfl_sync(kFull, kept, ql);
                const int n1 = __shfl_sync(kFull, kept, ql1 & 31);
                const bool two = n0 <= 16 && ql1 < nqc && !((spill_mask >> ql1) & 1u) && n1 <= 16;
                const int hw = two ? 16 : 32;   // lanes per row
                const int row = two ? ql + (lane >> 4) : ql;
                const int hl = two ? (lane & 15) : lane;
                const int n = two ? (lane >> 4 ? n1 : n0) : n0;
                const int width = two ? max(n0, n1) : n0;
                uint64_t key = ~0ull;
                if (hl < n) key = make_key(w.Ld[row * kListStr + hl], w.Li[row * kListStr + hl]);
#pragma unroll
                for (int k2 = 2; k2 <= 32; k2 <<= 1) {
                    if ((k2 >> 1) >= width) break;
#pragma unroll
                    for (int jj = k2 >> 1; jj > 0; jj >>= 1) {
                        const uint64_t other = __shfl_xor_sync(kFull, key, jj);
                        const bool take_min = ((hl & jj) == 0) == ((hl & k2) == 0);
                        key = (take_min == (other < key)) ? other : key;
                    }
                }
                const int cK = min(n, K);
                const int qo = __shfl_sync(kFull, qorig, row);
                int32_t* irow = oidx + (int64_t)qo * rstride_out;
                float* drow = od2 + (int64_t)qo * rstride_out;
                if (hl < cK) {
                    irow[hl] = (int32_t)(uint32_t)key;
                    drow[hl] = __uint_as_float((uint32_t)(key >> 32));
                } else if (!a.csr && hl < K) {
                    irow[hl] = -1;
                    drow[hl] = INFINITY;
                }
                for (int e2 = hw + hl; e2 < K && !a.csr; e2 += hw) {
                    irow[e2] = -1;
                    drow[e2] = INFINITY;
                }
                ql += two ? 2 : 1;
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------- overflow path
// Exact selection for queries with more than kListCap neighbours (whether or
// not that exceeds K): one warp per query scans the query's own +-m
// neighbourhood with lanes over candidates, appends keys below the current
// threshold to a shared buffer, and whenever the buffer is nearly full sorts
// it and keeps the K smallest (the threshold becomes the K-th key).  Keys are
// unique (indices differ), so the K smallest are unique.  The kernel always
// follows the grid query on its stream; its last block to finish clears the
// query's chunk counter (and, unless a compact fill pass still needs the
// overflow list, the list) for the next query, so no host-side memset
// interrupts the chain of programmatically dependent launches.

constexpr int kOvfWarps = 4;

__device__ void smem_bitonic(uint64_t* buf, int n) {
    const int lane = threadIdx.x & 31;
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncwarp();
            for (int i = lane; i < n / 2; i += 32) {
                const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                const int hi = lo + j;
                const bool up = (lo & k) == 0;
                const uint64_t x = buf[lo], y = buf[hi];
                if ((x > y) == up) {
                    buf[lo] = y;
                    buf[hi] = x;
                }
            }
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kOvfWarps * 32) k_overflow(QueryArgs a, int cap) {
    pdl_trigger();
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_o[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* buf = reinterpret_cast<uint64_t*>(smem_o) + (size_t)warp * cap;
    const int nov = min(*a.ovf_count, a.ovf_cap);
    const int D = a.D, K = a.K;
    const int DP = padded_dim(D);
    for (int w = blockIdx.x * kOvfWarps + warp; w < nov; w += gridDim.x * kOvfWarps) {
        const Overflow o = a.ovf[w];
        const EventHdr& h = a.ev[o.ev];
        int32_t* oidx = a.counts ? a.idx : h.idx;
        float* od2 = a.counts ? a.dist2 : h.dist2;
        const int qs = o.qslot;
        const int qo = a.qperm[qs];
        float qv[kMaxD];
#pragma unroll
        for (int k = 0; k < kMaxD; ++k) qv[k] = k < D ? a.qpts[pt_index(qs, k, DP)] : 0.f;
        const int qc = a.qcell[qs];
        const int dims0 = h.dims[0], m = h.m;
        const int x = qc % dims0, qrow = qc / dims0;
        const int self_slot = a.self ? qs : -1;
        const bool count_only = a.ovf_mode == 1;
        int fill = 0;
        int64_t deg = 0;
        uint64_t thr = ~0ull;
        for (int i = lane; i < cap && !count_only; i += 32) buf[i] = ~0ull;
        __syncwarp();
        const int nrows = neighbour_rows(h);
        for (int nr = 0; nr < nrows; ++nr) {
            int64_t rowbase;
            if (!neighbour_row(h, qrow, nr, rowbase)) continue;
            {
                const int rs = a.cstart[rowbase + max(x - m, 0)];
                const int re = a.cstart[rowbase + min(x + m, dims0 - 1) + 1];
                for (int c0 = rs; c0 < re; c0 += 32) {
                    const int cs = c0 + lane;
                    uint64_t key = ~0ull;
                    if (cs < re && cs != self_slot) {
                        float s = 0.f;
#pragma unroll
                        for (int k = 0; k < kMaxD; ++k) {
                            if (k < D) {
                                const float d = __fsub_rn(qv[k], a.rpts[pt_index(cs, k, DP)]);
                                s = __fadd_rn(s, __fmul_rn(d, d));
                            }
                        }
                        if (s <= a.r2) {
                            ++deg;
                            if (!count_only) {
                                key = make_key(s, a.rperm[cs]);
                                if (key >= thr) key = ~0ull;
                            }
                        }
                    }
                    if (count_only) continue;
                    const unsigned bal = __ballot_sync(kFull, key != ~0ull);
                    if (key != ~0ull) buf[fill + __popc(bal & ((1u << lane) - 1u))] = key;
                    fill += __popc(bal);
                    if (fill > cap - 32) {
                        smem_bitonic(buf, cap);
                        for (int i = K + lane; i < cap; i += 32) buf[i] = ~0ull;
                        fill = K;
                        thr = buf[K - 1];
                        __syncwarp();
                    }
                }
            }
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) deg += __shfl_xor_sync(kFull, deg, o2);
        const int32_t c = (int32_t)(deg < K ? deg : K);
        if (count_only) {
            // compact output, first pass: the row's count (marked) and degree
            if (lane == 0) {
                (a.counts ? a.counts : h.counts)[qo] = c | kCsrSpill;
                if (a.degree) a.degree[qo] = (int32_t)(deg < INT32_MAX ? deg : INT32_MAX);
            }
            continue;
        }
        const bool csr_rows = a.ovf_mode == 2;
        // a compact output too small for the rows (its caller fails the
        // call) is not written past its end
        if (csr_rows && a.row_off[qo] + c > a.row_cap) continue;
        smem_bitonic(buf, cap);
        int32_t* irow = oidx + (csr_rows ? a.row_off[qo] : (int64_t)qo * K);
        float* drow = od2 + (csr_rows ? a.row_off[qo] : (int64_t)qo * K);
        for (int e = lane; e < (csr_rows ? c : K); e += 32) {
            const uint64_t v = buf[e];
            const bool real = v != ~0ull;
            irow[e] = real ? (int32_t)(uint32_t)v : -1;
            drow[e] = real ? __uint_as_float((uint32_t)(v >> 32)) : INFINITY;
        }
        if (lane == 0 && !csr_rows) (a.counts ? a.counts : h.counts)[qo] = c;
        __syncwarp();
    }
    // the last block to finish clears the query's counters for the next launch
    __syncthreads();
    if (threadIdx.x == 0 && a.ovf_done) {
        __threadfence();
        if (atomicAdd(a.ovf_done, 1) == (int)gridDim.x - 1) {
            *a.task_counter = 0;
            if (a.reset_ovf) *a.ovf_count = 0;
            __threadfence();
            *a.ovf_done = 0;
        }
    }
}

// ------------------------------------------------------------- host launch

template <int D, int STAGE>
static cudaError_t launch_grid_query_ds(const QueryArgs& a, int num_sms, cudaStream_t st) {
    using C = QCfg<D, STAGE>;
    static_assert(C::TILE % 32 == 0, "whole lane rounds per tile");
    static_assert(C::NB <= 4, "phase bits and barriers per warp");
    static_assert(warp_smem_bytes<D, STAGE>() % 128 == 0 &&
                      (C::TILE * C::DP * sizeof(float)) % 16 == 0 && (C::DP * sizeof(float)) % 16 == 0,
                  "bulk-copy destinations and sizes must be 16-byte multiples");
    const size_t smem = (size_t)kQueryWarps * warp_smem_bytes<D, STAGE>();
    auto kern = &k_grid_query<D, STAGE>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (ce != cudaSuccess) return ce;
    int per_sm = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kQueryWarps * 32, smem);
    if (ce != cudaSuccess) return ce;
    per_sm = std::max(per_sm, 1);
    const int64_t warps = (int64_t)num_sms * per_sm * kQueryWarps;
    const int64_t blocks = std::max<int64_t>(
        1, std::min<int64_t>((int64_t)num_sms * per_sm,
                             ceil_div(std::min<int64_t>(a.nchunks, warps), kQueryWarps)));
    launch_pdl(kern, dim3((unsigned)blocks), dim3(kQueryWarps * 32), smem, st, a);
    return cudaGetLastError();
}

template <int D>
static cudaError_t launch_grid_query_d(const QueryArgs& a, int stage, int num_sms, cudaStream_t st) {
    return stage == kStageBulk ? launch_grid_query_ds<D, kStageBulk>(a, num_sms, st)
                               : launch_grid_query_ds<D, kStageLoads>(a, num_sms, st);
}

static QueryArgs query_args(const QueryLaunch& q) {
    const GridBufs& qs = *q.qset;
    const GridBufs& rs = *q.rset;
    QueryArgs a{};
    a.ev = rs.hdr;
    a.qev = qs.hdr;
    a.nev = qs.E;
    a.nchunks = (int32_t)(q.chunk_end >= 0 ? std::min<int64_t>(q.chunk_end, qs.nchunks) : qs.nchunks);
    a.qpts = qs.pts;
    a.qperm = qs.perm;
    a.qcell = qs.cell;
    a.rpts = rs.pts;
    a.rperm = rs.perm;
    a.cstart = rs.cstart;
    a.counts = q.counts;
    a.idx = q.idx;
    a.dist2 = q.dist2;
    a.r2 = q.r2;
    a.K = q.K;
    a.self = q.self;
    a.D = rs.D;
    a.task_counter = qs.scalars + kScTaskCounter;
    a.status = q.d_status;
    a.ovf = qs.ovf;
    a.ovf_count = qs.scalars + kScOvfCount;
    a.ovf_cap = (int32_t)std::max<int64_t>(qs.n_total, 1);
    a.ovf_done = qs.scalars + kScOvfDone;
    a.reset_ovf = q.ovf_mode == 1 ? 0 : 1;
    a.exit_dims = q.exit_dims;
    a.path_filter = q.path_filter;
    a.csr = q.csr;
    a.ovf_mode = q.ovf_mode;
    a.degree = q.degree;
    a.row_off = q.row_off;
    a.row_cap = q.row_cap;
    return a;
}

frnn_status enqueue_grid_query(const QueryLaunch& q, cudaStream_t st, std::string& err) {
    const GridBufs& qs = *q.qset;
    const GridBufs& rs = *q.rset;
    const QueryArgs a = query_args(q);
    // the chunk counter is zero here: the build clears it, and every query's
    // selection kernel clears it again when done.  The overflow list is
    // cleared the same way, except after a compact count pass whose fill pass
    // did not run.
    if (qs.ovf_stale) cudaMemsetAsync(qs.scalars + kScOvfCount, 0, sizeof(int32_t), st);
    qs.ovf_stale = q.ovf_mode == 1;
    if (q.kev[0]) cudaEventRecord(q.kev[0], st);
    cudaError_t ce = cudaSuccess;
    if (q.kernel == 1) {
        // grids of up to four axes: the row-task kernel (query_rows.cu)
        const frnn_status s = enqueue_row_query(q, a, st, err);
        if (s != FRNN_OK) return s;
    } else if (a.nchunks > 0) {
        switch (rs.D) {
#define FRNN_CASE(d) case d: ce = launch_grid_query_d<d>(a, q.stage, q.num_sms, st); break;
            FRNN_CASE(1) FRNN_CASE(2) FRNN_CASE(3) FRNN_CASE(4) FRNN_CASE(5) FRNN_CASE(6)
            FRNN_CASE(7) FRNN_CASE(8) FRNN_CASE(9) FRNN_CASE(10) FRNN_CASE(11) FRNN_CASE(12)
            FRNN_CASE(13) FRNN_CASE(14) FRNN_CASE(15) FRNN_CASE(16)
#undef FRNN_CASE
            default:
                err = "unsupported D";
                return FRNN_ERR_INVALID_ARG;
        }
    }
    if (ce != cudaSuccess) {
        err = std::string("grid query launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    if (q.kev[1]) cudaEventRecord(q.kev[1], st);
    return enqueue_overflow(a, q.num_sms, st, err);
}

frnn_status enqueue_overflow_only(const QueryLaunch& q, cudaStream_t st, std::string& err) {
    QueryArgs o = query_args(q);
    o.path_filter = -1;
    o.reset_ovf = 1;   // the fill pass consumes the list
    q.qset->ovf_stale = false;
    return enqueue_overflow(o, q.num_sms, st, err);
}

frnn_status enqueue_overflow(const QueryArgs& a, int num_sms, cudaStream_t st, std::string& err) {
    // buffer of a power of two >= 2K keys per warp
    int cap = 64;
    while (cap < 2 * a.K) cap <<= 1;
    const size_t osmem = (size_t)kOvfWarps * cap * sizeof(uint64_t);
    cudaError_t ce =
        cudaFuncSetAttribute(k_overflow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osmem);
    if (ce == cudaSuccess) {
        launch_pdl(k_overflow, dim3(num_sms), dim3(kOvfWarps * 32), osmem, st, a, cap);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) {
        err = std::string("selection kernel launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    return FRNN_OK;
}

}  // namespace frnn
