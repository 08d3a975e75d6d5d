// query_rows.cu — the grid scan for grids of up to four gridded axes: warp
// tasks of 16 cell-sorted queries in one row of cells, the union of their
// neighbour rows streamed through shared memory by bulk copies and screened
// against all 16 queries at once, an exact float32 recheck and warp-level
// top-K.  (Grids of five axes, whose cells hold few points, use the chunk
// kernel of query.cu; the library picks by the requested axis count.)
//
// Method (Eq. 1, Sec. 1): for each query, every reference in the cells within
// +-m cells along each gridded axis is a candidate (complete by the grid's
// roundoff-safe construction, build.cu); each candidate's squared distance is
// computed under the fixed float32 contract and kept if <= fl(r*r).
//
// Organisation on the GPU (differs from the paper's thread-per-query kernel,
// whose profile showed dependent-load latency and divergence, Sec. 4.2):
//   * a persistent grid; each warp takes warp tasks (16 cell-sorted queries in
//     one row of cells) from an atomic counter; lanes q and q + 16 serve query
//     q and split the candidates between them (even and odd pairs), so a warp
//     screens the union of 16 neighbourhoods, not 32: fewer candidates per
//     query (the union of a longer run of queries spans more cells);
//   * the candidates of a task are the union of its lanes' neighbourhoods: per
//     neighbour row one contiguous slot range; the ranges, widened to pair
//     boundaries, form one stream of candidate pairs cut into tiles of TILEP
//     pairs; the row lanes copy their parts of a tile into the warp's
//     shared-memory ring with cp.async.bulk, completion tracked by one
//     mbarrier per buffer (prefetch depth NBUF-1); once the last tile is
//     consumed the ring is reused for the lists' distances;
//   * every lane screens every candidate of the tile (broadcast shared loads):
//     warp-uniform control flow.  Points are stored pair-interleaved, so each
//     16-byte shared load gives two dimensions of two candidates and one
//     packed f32x2 instruction serves two candidates.  The packed arithmetic
//     is only a conservative screen (proof below);
//   * early rejection: after the first `EXIT` dimensions the warp votes;
//     partial sums never decrease (round-to-nearest of non-negative terms), so
//     if every lane's partial sum already exceeds the screen bound the
//     candidate is rejected for all of them without changing any verdict (the
//     paper's "roundoff-safe early rejection", Sec. 6).  Gridded axes are the
//     last ones by default, so the first dimensions are ungridded, the most
//     selective ones;
//   * a candidate that passes the whole screen is appended to the lane's list
//     in shared memory as its stream position; at the end of the task the
//     warp resolves every lane's entries together (row, slot, range filter)
//     and recomputes each with the scalar contract, which alone decides
//     membership and gives the distance (the paper's "conservative screening
//     and canonical-order recomputation", Sec. 4.2); the original index is
//     looked up only for the kept entries (the deferred lookup, Table 3);
//   * for each query the warp loads its lanes' entries (at most 32, one per
//     lane), sorts them by (d2, index) with a bitonic network across the lanes
//     (shuffles), and writes the first K (count = min(degree, K)) coalesced,
//     with the padding.  Lists longer than 32 go to the exact selection
//     kernel of query.cu, keeping results exact for dense inputs (the paper's
//     Sec. 5 caveat on heap-free top-K).
#include <algorithm>
#include <cmath>

#include "frnn_host.h"

namespace frnn {
namespace rows {

// This kernel reads the cell-sorted points pair-interleaved: slots 2p and
// 2p+1 share a block of 2*DP floats [s0.d0, s1.d0, s0.d1, s1.d1, ...], so one
// 16-byte load yields two dimensions of two candidates, the operand layout
// of the packed f32x2 screen.  The copy is made from the plain rows at query
// time (k_pack_pairs); every event starts on an even slot.
__host__ __device__ constexpr int64_t pair_index(int64_t slot, int k, int DP) {
    return (slot >> 1) * 2 * DP + 2 * k + (slot & 1);
}

constexpr int kQueryWarps = 4;
constexpr int kMaxNBuf = 4;
// candidate streams per query: lanes q, q + G, q + 2G, ... (G = queries per
// warp task) serve query q, each taking every kStreams-th candidate pair
constexpr int kStreams = 32 / kTaskQueries;
static_assert(kStreams * kTaskQueries == 32, "the lanes of a warp split evenly");
constexpr uint32_t kFull = 0xffffffffu;
// per-lane list in shared memory: a lane holds about half of its query's
// entries, so 24 rarely overflows (an overflow only sends the row to the
// selection kernel) and the smaller lists let seven CTAs share an SM
constexpr int kListCap = 24;
constexpr int kRowCap = 32;       // entries of one query sorted across the warp (one per lane)
constexpr int kListStride = 33;   // entry e of lane l at e*33 + l: conflict-free both ways
static_assert(kRowCap <= kCsrStageW, "a staged compact row holds a whole row");

template <int D>
struct QCfg {
    static constexpr int DP = padded_dim(D);
    // candidate pairs per tile, ring buffers and CTAs per SM.  The ring (two
    // tiles) doubles as the list distances once the tiles are consumed, so up
    // to D = 8 a warp needs under 8 KB of shared memory and seven CTAs (28
    // warps, at most 72 registers) share an SM, which the latency-bound scan
    // prefers.  Measured at 300k x 8 (before the warp-wide row sort): 2 KB
    // tiles with six CTAs 0.292 ms, 1 KB tiles 0.310 (0.321 with five CTAs),
    // 3 KB tiles with five CTAs 0.298; after it, seven CTAs 0.266 against six
    // 0.270.  At 500k x 12: 3 KB tiles 0.493 ms, 2.25 KB 0.512, 1.5 KB 0.548.
    static constexpr int TILEP = DP == 4 ? 64 : (DP == 8 ? 32 : (DP == 12 ? 32 : 16));
    static constexpr int MINB = DP <= 8 ? 7 : 4;
    static constexpr int NBUF = 2;
    // default vote point (measured: 2 and 3 tie at D = 8, 3 is best at D = 12)
    static constexpr int EXIT = D <= 4 ? D : (D >= 10 ? 3 : 2);
    // sort two short query rows at once, one per half-warp.  Measured: 500k x
    // 12 (about 12 neighbours per clustered query) 0.437 -> 0.424 ms; at 300k
    // x 8 (about 25, rows rarely pair) the paired loop cost 0.8 %, so lower
    // dimensions keep the one-row loop
    static constexpr bool PAIR_ROWS = D >= 10;
};

__host__ __device__ constexpr size_t ring_floats(int DP, int TILEP, int NB) {
    return (size_t)NB * TILEP * 2 * DP;
}
__host__ __device__ constexpr size_t warp_smem_bytes(int DP, int TILEP, int NB);
__host__ __device__ constexpr size_t query_smem_bytes(int DP, int TILEP, int NB) {
    return (size_t)kQueryWarps * warp_smem_bytes(DP, TILEP, NB);
}

// ------------------------------------------------------------- packed f32x2
// Two float32 lanes per instruction.  The assembler contracts packed
// multiply/add pairs into fused multiply-adds whatever the flags (measured), so
// packed arithmetic is used ONLY for a conservative screen: for any subset of
// k <= 16 dimensions, fused or unfused rounding keeps the packed partial sum
// s' within (1 +- 2^-24)^(2k) of the exact sum S of the same rounded squared
// differences, and the contract's full sum s_D >= S (1 - 2^-24)^(2D).  Hence
// s' > r2 (1 + 2^-16) implies s_D > r2: rejecting there never drops a pair.
// Every candidate that survives is recomputed with the scalar contract
// (__fsub_rn / __fmul_rn / __fadd_rn, never contracted), which decides
// membership and gives the returned distance (the paper's "conservative
// screening and canonical-order recomputation", Sec. 4.2).

__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// screening step for two candidates: s' += (q - c)^2 (fused)
__device__ __forceinline__ uint64_t f2_screen(uint64_t s, uint64_t q, uint64_t c) {
    const uint64_t d = f2_sub(q, c);
    return f2_fma(d, d, s);
}

__device__ __forceinline__ uint64_t make_key(float d2, int32_t j) {
    return ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)j;
}

// ------------------------------------------------------------- grid query

// Per-warp shared memory: the tile ring, the per-lane lists, the task's
// neighbour-row table, per-lane accept counters and the ring's mbarriers.
struct WarpSmem {
    float* ring;
    float* Ld;
    int32_t* Li;
    int32_t* Rpp;    // [32] first stream pair of neighbour row l
    int32_t* Rprs;   // [32] its first pair in slot space
    int32_t* Rrs;    // [32] its slot range [rs, re)
    int32_t* Rre;
    int32_t* acc;    // [32] exactly accepted entries per lane
    uint64_t* bars;  // [NBUF]
};

// The ring and the lists' distances share one region (the distances are
// written only after the last tile is consumed).  Rounded up to 128 bytes:
// every warp's ring (a bulk-copy destination) must start on a 16-byte
// boundary.
__host__ __device__ constexpr size_t ring_region_floats(int DP, int TILEP, int NB) {
    return ring_floats(DP, TILEP, NB) > (size_t)kListCap * kListStride
               ? ring_floats(DP, TILEP, NB)
               : (size_t)kListCap * kListStride;
}
__host__ __device__ constexpr size_t warp_smem_bytes(int DP, int TILEP, int NB) {
    return (ring_region_floats(DP, TILEP, NB) * sizeof(float) + kListCap * kListStride * 4 +
            5 * 32 * 4 + NB * sizeof(uint64_t) + 127) / 128 * 128;
}

__device__ __forceinline__ WarpSmem carve_warp(unsigned char* base, int DP, int TILEP, int NB) {
    WarpSmem w;
    w.ring = reinterpret_cast<float*>(base);
    w.Ld = w.ring;   // after the tiles
    w.Li = reinterpret_cast<int32_t*>(w.ring + ring_region_floats(DP, TILEP, NB));
    w.Rpp = w.Li + kListCap * kListStride;
    w.Rprs = w.Rpp + 32;
    w.Rrs = w.Rprs + 32;
    w.Rre = w.Rrs + 32;
    w.acc = w.Rre + 32;
    w.bars = reinterpret_cast<uint64_t*>(w.acc + 32);
    return w;
}

// One warp task: 16 queries in one row of cells; their candidates are the
// slot ranges of the neighbour rows (lane l < neighbour_rows owns row l),
// each widened to pair boundaries and concatenated into one stream of
// candidate pairs.  Tile t of the stream (TILEP pairs) may span several rows:
// every row lane that overlaps it copies its own part with cp.async.bulk,
// all completing on the buffer's one mbarrier.  A tentative entry is stored
// as its stream code 2 * pair + half; the row it came from, its slot, the
// row-range filter and the exact recheck are resolved at the end of the task.
template <int TILEP, int PAIRF>
__device__ __forceinline__ void issue_tile(const WarpSmem& w, int t, int b, int pp, int np,
                                           int prs, int P, const float* rpts, int lane) {
    const int T0 = t * TILEP;
    const int T1 = min(T0 + TILEP, P);
    if (lane == 0)
        mbar_arrive_expect_tx(&w.bars[b], (uint32_t)(T1 - T0) * PAIRF * sizeof(float));
    __syncwarp();
    const int lo_s = max(pp, T0), hi_s = min(pp + np, T1);
    if (hi_s > lo_s) {
        fence_proxy_async_smem();   // the buffer's previous contents were read generically
        bulk_g2s(w.ring + (size_t)b * TILEP * PAIRF + (size_t)(lo_s - T0) * PAIRF,
                 rpts + (int64_t)(prs + lo_s - pp) * PAIRF,
                 (uint32_t)(hi_s - lo_s) * PAIRF * sizeof(float), &w.bars[b]);
    }
}

template <int D, int EXIT>
__global__ void __launch_bounds__(kQueryWarps * 32, QCfg<D>::MINB) k_row_query(QueryArgs a) {
    pdl_trigger();
    pdl_wait();
    using C = QCfg<D>;
    constexpr int DP = C::DP;
    constexpr int TILEP = C::TILEP;
    constexpr int PAIRF = 2 * DP;   // floats per candidate pair
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NB = C::NBUF;
    const WarpSmem w =
        carve_warp(smem + (size_t)warp * warp_smem_bytes(DP, TILEP, NB), DP, TILEP, NB);
    float* Ld = w.Ld;
    int32_t* Li = w.Li;
    // lanes q, q + G, ... serve the task's query q (G = kTaskQueries); lane
    // q + s G screens the candidate pairs p with p mod kStreams == s
    const int qi = lane % kTaskQueries;
    const int sh = lane / kTaskQueries;
    if (lane == 0)
        for (int b = 0; b < NB; ++b) mbar_init(&w.bars[b], 1);
    fence_mbar_init();
    __syncwarp();
    uint32_t phase = 0;   // bit b: parity to wait for on buffer b

    const int ntasks = *a.ntasks;
    const float r2 = a.r2;
    const float rs2 = a.r2_screen;
    const int K = a.K;

    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.task_counter, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= ntasks) break;
        const Task task = a.tasks[t];
        const EventHdr& h = a.ev[task.ev];
        if (a.path_filter >= 0 && h.path != a.path_filter) continue;   // another launch's event
        int32_t* counts = a.counts ? a.counts : h.counts;
        int32_t* oidx = a.counts ? a.idx : h.idx;
        float* od2 = a.counts ? a.dist2 : h.dist2;

        const bool act = qi < task.nq;
        const int qs = task.qslot + qi;
        const int qorig = act ? a.qperm[qs] : 0;
        if (!h.valid) {
            // grid built from non-finite input: empty rows (frnn_sync reports it)
            for (int ql = 0; ql < task.nq && !a.csr; ++ql) {
                const int qo = __shfl_sync(kFull, qorig, ql);
                for (int e = lane; e < K; e += 32) {
                    oidx[(int64_t)qo * K + e] = -1;
                    od2[(int64_t)qo * K + e] = INFINITY;
                }
            }
            if (act && sh == 0) counts[qorig] = 0;
            if (act && sh == 0 && a.degree) a.degree[qorig] = 0;
            continue;
        }
        uint64_t qq[D];   // each query coordinate duplicated into both f32x2 lanes
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float v = act ? a.qpts[pair_index(qs, k, DP)] : __int_as_float(0x7fc00000);
            qq[k] = f2_pack(v, v);   // inactive lanes: NaN, never within r
        }
        const int qc = act ? a.qcell[qs] : 0;
        const int dims0 = h.dims[0], m = h.m;
        const int x = qc % dims0;
        const int xa = __shfl_sync(kFull, x, 0);
        const int xb = __shfl_sync(kFull, x, task.nq - 1);

        // neighbour row of this lane (lane < neighbour_rows <= 32) and its
        // place in the candidate stream
        const int nrows = neighbour_rows(h);
        int rs = 0, re = 0;
        int64_t rowbase;
        if (lane < nrows && neighbour_row(h, task.row, lane, rowbase)) {
            const int x0 = max(xa - m, 0), x1 = min(xb + m, dims0 - 1);
            rs = a.cstart[rowbase + x0];
            re = a.cstart[rowbase + x1 + 1];
        }
        const int prs = rs >> 1;
        const int np = re > rs ? ((re + 1) >> 1) - prs : 0;
        int incl = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const int pp = incl - np;
        const int P = __shfl_sync(kFull, incl, 31);
        w.Rpp[lane] = pp;   // nondecreasing over lanes (empty rows repeat the next start)
        w.Rprs[lane] = prs;
        w.Rrs[lane] = rs;
        w.Rre[lane] = re;
        w.acc[lane] = 0;
        // the query's own slot lies in the centre row (every offset zero); in
        // a self-query it is excluded by its stream code
        const int lc = (nrows - 1) >> 1;
        const int pp_c = __shfl_sync(kFull, pp, lc), prs_c = __shfl_sync(kFull, prs, lc);
        const int self_code = (a.self && act) ? 2 * (pp_c + (qs >> 1) - prs_c) + (qs & 1) : -1;
        const int ntiles = (P + TILEP - 1) / TILEP;

        int cnt = 0;          // tentative entries (more than kListCap: the row goes to the selection kernel)

        // prologue: fill the ring
        const int pre = min(NB, ntiles);
        for (int tt = 0; tt < pre; ++tt)
            issue_tile<TILEP, PAIRF>(w, tt, tt, pp, np, prs, P, a.rpts, lane);
        int timed_out_at = -1;
        for (int tt = 0; tt < ntiles; ++tt) {
            const int b = tt % NB;
            if (!mbar_wait_bounded(&w.bars[b], (phase >> b) & 1u)) {
                timed_out_at = tt;
                break;
            }
            phase ^= 1u << b;
            float* tile = w.ring + (size_t)b * TILEP * PAIRF;
            const int T0 = tt * TILEP;
            const int lenp = min(TILEP, P - T0);
            {
                // a row whose slot range starts (ends) inside a pair: put NaN
                // into the first coordinate of the half outside the range, so
                // it fails every screen (the neighbouring slot belongs to a
                // cell outside the search range, or to another row's part)
                const int lo_s = max(pp, T0), hi_s = min(pp + np, T0 + lenp);
                if (hi_s > lo_s && (((lo_s == pp) && (rs & 1)) || ((hi_s == pp + np) && (re & 1)))) {
                    if (lo_s == pp && (rs & 1)) tile[(lo_s - T0) * PAIRF] = __int_as_float(0x7fc00000);
                    if (hi_s == pp + np && (re & 1))
                        tile[(hi_s - 1 - T0) * PAIRF + 1] = __int_as_float(0x7fc00000);
                    fence_proxy_async_smem();   // before the buffer is refilled by bulk copies
                }
                // the last tile of the task: the pairs between its end and the
                // end of the last screening step hold stale data; NaN makes
                // them fail every screen (both halves)
                const int pend = (lenp + 4 * kStreams - 1) / (4 * kStreams) * (4 * kStreams);
                if (lane < pend - lenp) {
                    float* f = tile + (size_t)(lenp + lane) * PAIRF;
                    f[0] = __int_as_float(0x7fc00000);
                    f[1] = __int_as_float(0x7fc00000);
                    fence_proxy_async_smem();
                }
                __syncwarp();
            }
            // four candidate pairs per stream and step: their first-stage
            // screens are independent, which hides the packed pipeline's
            // latency
            for (int p0 = 0; p0 < lenp; p0 += 4 * kStreams) {
                uint64_t sg[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int p = p0 + kStreams * j + sh;
                    const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(tile + p * PAIRF);
                    uint64_t s2 = 0;
#pragma unroll
                    for (int k = 0; k < EXIT; ++k) {
                        const ulonglong2 v = cp[k >> 1];
                        s2 = f2_screen(s2, qq[k], (k & 1) ? v.y : v.x);
                    }
                    sg[j] = s2;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int p = p0 + kStreams * j + sh;
                    const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(tile + p * PAIRF);
                    uint64_t s2 = sg[j];
                    float s0, s1;
                    f2_unpack(s2, s0, s1);
                    if (!__any_sync(kFull, fminf(s0, s1) <= rs2)) continue;
                    if (EXIT < D) {
#pragma unroll
                        for (int k = EXIT; k < D; ++k) {
                            const ulonglong2 v = cp[k >> 1];
                            s2 = f2_screen(s2, qq[k], (k & 1) ? v.y : v.x);
                        }
                        f2_unpack(s2, s0, s1);
                    }
                    // tentative entries: the stream codes, resolved at the task's
                    // end; appended without branches (predicated stores), so the
                    // warp does not diverge here
                    const int code0 = 2 * (T0 + p);
                    const bool f0 = s0 <= rs2 && code0 != self_code;
                    const bool f1 = s1 <= rs2 && code0 + 1 != self_code;
                    const int c1 = cnt + (f0 ? 1 : 0);
                    if (f0 && cnt < kListCap) Li[cnt * kListStride + lane] = code0;
                    if (f1 && c1 < kListCap) Li[c1 * kListStride + lane] = code0 + 1;
                    cnt = c1 + (f1 ? 1 : 0);
                }
            }
            __syncwarp();
            const int nt = tt + NB;
            if (nt < ntiles) issue_tile<TILEP, PAIRF>(w, nt, b, pp, np, prs, P, a.rpts, lane);
        }
        if (timed_out_at >= 0) {
            // record, wait (bounded) for the copies still in flight, stop this warp
            if (lane == 0) atomicOr(a.status, kStatusTimeout);
            const int issued = min(ntiles, timed_out_at + NB);
            for (int t2 = timed_out_at; t2 < issued; ++t2) {
                const int b2 = t2 % NB;
                mbar_wait_bounded(&w.bars[b2], (phase >> b2) & 1u);
                phase ^= 1u << b2;
            }
            return;
        }

        const bool lost = cnt > kListCap;   // an entry did not fit the list
        // exact recheck of every lane's tentative entries, spread over the
        // whole warp: entry i of the task's concatenated lists goes to lane
        // i % 32.  Each resolves its row (the last row whose stream part
        // starts at or before the pair), its slot and the row-range filter
        // (slots read only because parts start on pair boundaries are
        // dropped), then applies the scalar contract in index order without
        // contraction.  Accepted: (d2, slot); rejected: d2 = +inf, sorted last.
        const int own = lost ? 0 : cnt;
        int cin = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, cin, o);
            if (lane >= o) cin += v;
        }
        const int cex = cin - own;
        const int T = __shfl_sync(kFull, cin, 31);
        __syncwarp();
        for (int base = 0; base < T; base += 32) {
            const int i = base + lane;
            // owner lane: the last lane whose entries start at or before i
            int O = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int v = __shfl_sync(kFull, cex, O + st);
                if (v <= i) O += st;
            }
            const int e = i - __shfl_sync(kFull, cex, O);
            if (i < T) {
                const int code = Li[e * kListStride + O];
                const int sp = code >> 1;
                int L = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1)
                    if (w.Rpp[L + st] <= sp) L += st;
                const int slot = 2 * (w.Rprs[L] + sp - w.Rpp[L]) + (code & 1);
                float sv = INFINITY;
                int32_t orig = 0;
                if (slot >= w.Rrs[L] && slot < w.Rre[L]) {
                    orig = a.rperm[slot];   // in flight with the coordinate loads
                    const int qo_slot = task.qslot + (O % kTaskQueries);
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float d = __fsub_rn(a.qpts[pair_index(qo_slot, k, DP)],
                                                  a.rpts[pair_index(slot, k, DP)]);
                        acc = __fadd_rn(acc, __fmul_rn(d, d));
                    }
                    if (acc <= r2) {
                        sv = acc;
                        atomicAdd(&w.acc[O], 1);
                    }
                }
                Ld[e * kListStride + O] = sv;
                Li[e * kListStride + O] = sv <= r2 ? orig : 0;   // rejected: +inf sorts last
            }
        }
        __syncwarp();
        const int kept = w.acc[lane];
        // per query: its lanes' entries together (rejected ones carry +inf)
        int cnt_q = cnt, kept_q = kept;
        bool lost_q = lost;
#pragma unroll
        for (int st = 1; st < kStreams; ++st) {
            cnt_q += __shfl_sync(kFull, cnt, qi + st * kTaskQueries);
            kept_q += __shfl_sync(kFull, kept, qi + st * kTaskQueries);
            lost_q |= __shfl_sync(kFull, lost, qi + st * kTaskQueries);
        }
        // more than 32 entries: the exact selection kernel finishes the row
        const bool spill = sh == 0 && act && (lost_q || cnt_q > kRowCap);
        if (sh == 0 && act && !spill) counts[qorig] = min(kept_q, K);
        if (spill && a.csr) counts[qorig] = kCsrSpill;   // counted by the selection kernel
        if (sh == 0 && act && !spill && a.degree) a.degree[qorig] = kept_q;
        if (spill) {
            const int pos = atomicAdd(a.ovf_count, 1);
            if (pos < a.ovf_cap) {
                a.ovf[pos].qslot = qs;
                a.ovf[pos].ev = task.ev;
            } else {
                atomicOr(a.status, kStatusCapacity);
            }
        }
        // one query row at a time (for D >= 10 two short rows at a time, one
        // per half-warp): lane l takes entry l of the query's lists, the warp
        // sorts the 32 keys (d2 bits << 32 | original index; unused lanes hold
        // the largest key) with a bitonic network across lanes, and lane l
        // writes position l of the row (coalesced), then the padding
        const unsigned spill_mask = __ballot_sync(kFull, spill);
        const int rstride = a.csr ? kCsrStageW : K;
        if constexpr (!C::PAIR_ROWS) {
            for (int ql = 0; ql < task.nq; ++ql) {
                if (spill_mask & (1u << ql)) continue;
                uint64_t key = ~0ull;
                int base = 0;
#pragma unroll
                for (int st = 0; st < kStreams; ++st) {
                    const int col = ql + st * kTaskQueries;
                    const int c = __shfl_sync(kFull, cnt, col);
                    if (lane >= base && lane < base + c)
                        key = make_key(Ld[(lane - base) * kListStride + col],
                                       Li[(lane - base) * kListStride + col]);
                    base += c;
                }
                // the network only as wide as the row needs (base entries sit in
                // lanes 0 .. base-1; wider stages would compare largest keys only)
#pragma unroll
                for (int k2 = 2; k2 <= 32; k2 <<= 1) {
                    if ((k2 >> 1) >= base) break;
#pragma unroll
                    for (int j = k2 >> 1; j > 0; j >>= 1) {
                        const uint64_t other = __shfl_xor_sync(kFull, key, j);
                        const bool take_min = ((lane & j) == 0) == ((lane & k2) == 0);
                        // one comparison: equal keys (rejected entries, empty lanes)
                        // are interchangeable, all others are distinct
                        key = (take_min == (other < key)) ? other : key;
                    }
                }
                const int c = min(__shfl_sync(kFull, kept_q, ql), K);
                const int qo = __shfl_sync(kFull, qorig, ql);
                int32_t* irow = oidx + (int64_t)qo * rstride;
                float* drow = od2 + (int64_t)qo * rstride;
                if (lane < c) {
                    irow[lane] = (int32_t)(uint32_t)key;
                    drow[lane] = __uint_as_float((uint32_t)(key >> 32));
                } else if (!a.csr && lane < K) {
                    irow[lane] = -1;
                    drow[lane] = INFINITY;
                }
                for (int e = 32 + lane; e < K && !a.csr; e += 32) {
                    irow[e] = -1;
                    drow[e] = INFINITY;
                }
            }
        } else {
            // two rows at a time, one per half-warp, when both hold at most
            // 16 entries (the network then stays within each half and both
            // halves end ascending); otherwise one row per warp as above
            for (int ql = 0; ql < task.nq;) {
                if (spill_mask & (1u << ql)) {
                    ++ql;
                    continue;
                }
                const int ql1 = ql + 1;   // <= 16: a valid lane
                const int n0 = __shfl_sync(kFull, cnt_q, ql);
                const int n1 = __shfl_sync(kFull, cnt_q, ql1);
                const bool two =
                    n0 <= 16 && ql1 < task.nq && !(spill_mask & (1u << ql1)) && n1 <= 16;
                const int hw = two ? 16 : 32;   // lanes per row
                const int row = two ? ql + (lane >> 4) : ql;
                const int hl = two ? (lane & 15) : lane;
                const int width = two ? max(n0, n1) : n0;
                uint64_t key = ~0ull;
                int base = 0;
#pragma unroll
                for (int st = 0; st < kStreams; ++st) {
                    const int col = row + st * kTaskQueries;
                    const int c = __shfl_sync(kFull, cnt, col);
                    if (hl >= base && hl < base + c)
                        key = make_key(Ld[(hl - base) * kListStride + col],
                                       Li[(hl - base) * kListStride + col]);
                    base += c;
                }
#pragma unroll
                for (int k2 = 2; k2 <= 32; k2 <<= 1) {
                    if ((k2 >> 1) >= width) break;
#pragma unroll
                    for (int j = k2 >> 1; j > 0; j >>= 1) {
                        const uint64_t other = __shfl_xor_sync(kFull, key, j);
                        const bool take_min = ((hl & j) == 0) == ((hl & k2) == 0);
                        key = (take_min == (other < key)) ? other : key;
                    }
                }
                const int c = min(__shfl_sync(kFull, kept_q, row), K);
                const int qo = __shfl_sync(kFull, qorig, row);
                int32_t* irow = oidx + (int64_t)qo * rstride;
                float* drow = od2 + (int64_t)qo * rstride;
                if (hl < c) {
                    irow[hl] = (int32_t)(uint32_t)key;
                    drow[hl] = __uint_as_float((uint32_t)(key >> 32));
                } else if (!a.csr && hl < K) {
                    irow[hl] = -1;
                    drow[hl] = INFINITY;
                }
                for (int e = hw + hl; e < K && !a.csr; e += hw) {
                    irow[e] = -1;
                    drow[e] = INFINITY;
                }
                ql += two ? 2 : 1;
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------- overflow path

}  // namespace rows

// ------------------------------------------------------------- preparation

// The pair-interleaved copy, one thread per slot pair (events start on even
// slots, so every pair lies inside one event).
__global__ void __launch_bounds__(256) k_pack_pairs(const float* pts, int64_t npairs, int DP,
                                                    float* ppts) {
    pdl_trigger();
    pdl_wait();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npairs) return;
    const float4* a = reinterpret_cast<const float4*>(pts + 2 * q * DP);
    const float4* b = reinterpret_cast<const float4*>(pts + (2 * q + 1) * DP);
    float4* dst = reinterpret_cast<float4*>(ppts + 2 * q * DP);
    for (int j = 0; j < DP / 4; ++j) {
        const float4 u = a[j], v = b[j];
        dst[2 * j] = make_float4(u.x, v.x, u.y, v.y);
        dst[2 * j + 1] = make_float4(u.z, v.z, u.w, v.w);
    }
}

static size_t al256r(size_t x) { return (x + 255) / 256 * 256; }

void rows_free(GridBufs& g) {
    if (g.rows_base) cudaFree(g.rows_base);
    g.rows_base = nullptr;
    g.rows_bytes = 0;
    g.rows_cap_n = g.rows_cap_tasks = g.rows_cap_L = 0;
    g.rows_cap_DP = 0;
    g.ppts = nullptr;
    g.row_tasks = nullptr;
    g.rows_rtask = nullptr;
    g.rows_ready = false;
}

frnn_status rows_reserve(GridBufs& g, std::string& err) {
    // a row of c queries opens ceil(c / 16) tasks: at most n / 16 + rows per event
    int64_t tcap = 0;
    for (int e = 0; e < g.E; ++e)
        tcap += g.h_hdr[e].n / kTaskQueries + std::min<int64_t>(g.h_hdr[e].cell_cap, g.h_hdr[e].n) + 2;
    if (tcap >= INT32_MAX) {
        err = "too many row tasks for one call";
        return FRNN_ERR_INVALID_ARG;
    }
    const int64_t n = std::max<int64_t>(g.n_total, 2);
    if (g.rows_base && g.rows_cap_n >= n && g.rows_cap_DP >= g.DP && g.rows_cap_tasks >= tcap &&
        g.rows_cap_L >= g.L)
        return FRNN_OK;
    rows_free(g);
    const size_t bp = al256r(sizeof(float) * (size_t)g.DP * (n + kTcRowPad));
    const size_t bt = al256r(sizeof(Task) * (size_t)tcap);
    const size_t br = al256r(sizeof(int32_t) * (size_t)std::max<int64_t>(g.L, 1));
    void* base = nullptr;
    if (cudaMalloc(&base, bp + bt + br) != cudaSuccess) {
        cudaGetLastError();
        err = "cudaMalloc of the row-task buffers failed";
        return FRNN_ERR_OUT_OF_MEMORY;
    }
    char* b = static_cast<char*>(base);
    g.rows_base = base;
    g.rows_bytes = bp + bt + br;
    g.ppts = reinterpret_cast<float*>(b);
    g.row_tasks = reinterpret_cast<Task*>(b + bp);
    g.rows_rtask = reinterpret_cast<int32_t*>(b + bp + bt);
    g.rows_cap_n = n;
    g.rows_cap_DP = g.DP;
    g.rows_cap_tasks = tcap;
    g.rows_cap_L = g.L;
    return FRNN_OK;
}

frnn_status rows_prepare(GridBufs& g, int32_t* d_status, cudaStream_t st, std::string& err,
                         int path_filter, int64_t i0, int64_t i1, int64_t s0, int64_t s1) {
    if (g.rows_ready) return FRNN_OK;
    frnn_status s = rows_reserve(g, err);
    if (s != FRNN_OK) return s;
    // slots of the events to prepare (event regions start on even slots)
    if (s1 < 0) s1 = g.n_total;
    s0 = std::min(std::max<int64_t>(s0, 0), s1) & ~(int64_t)1;
    const int64_t np = (s1 - s0) / 2;
    if (np > 0)
        launch_pdl(k_pack_pairs, dim3((unsigned)ceil_div(np, 256)), dim3(256), 0, st,
                   (const float*)g.pts + s0 * g.DP, np, g.DP, g.ppts + s0 * g.DP);
    g.rtask = g.rows_rtask;   // the task builder's scratch
    enqueue_tasks(g, kTaskQueries, 1, g.row_tasks, g.rows_cap_tasks, g.scalars + kScNTasks,
                  d_status, st, path_filter, i0, i1);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("row-task preparation failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    g.rows_ready = true;
    return FRNN_OK;
}

// ------------------------------------------------------------- launch

template <int D>
static cudaError_t launch_row_query_d(const QueryArgs& a, int exit_dims, int num_sms,
                                      cudaStream_t st) {
    using namespace rows;
    using C = QCfg<D>;
    static_assert(C::TILEP % (4 * kStreams) == 0, "whole screening steps per tile");
    static_assert(C::NBUF <= kMaxNBuf, "phase bits and barriers per warp");
    static_assert(warp_smem_bytes(C::DP, C::TILEP, C::NBUF) % 16 == 0 &&
                      (ring_region_floats(C::DP, C::TILEP, C::NBUF) * sizeof(float)) % 16 == 0 &&
                      (2 * C::DP * sizeof(float)) % 16 == 0,
                  "bulk-copy destinations and sizes must be 16-byte multiples");
    const size_t smem = query_smem_bytes(C::DP, C::TILEP, C::NBUF);
    auto kern = &k_row_query<D, C::EXIT>;
    // other vote points are compiled for the tracking-like dimensions only
    if constexpr (D == 8 || D == 12) {
        if (exit_dims == 1) kern = &k_row_query<D, 1>;
        else if (exit_dims == 2) kern = &k_row_query<D, 2>;
        else if (exit_dims == 3) kern = &k_row_query<D, 3>;
        else if (exit_dims == 4) kern = &k_row_query<D, 4>;
        else if (exit_dims >= 5) kern = &k_row_query<D, 6>;
    }
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (ce != cudaSuccess) return ce;
    int per_sm = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kQueryWarps * 32, smem);
    if (ce != cudaSuccess) return ce;
    per_sm = std::max(per_sm, 1);
    launch_pdl(kern, dim3(num_sms * per_sm), dim3(kQueryWarps * 32), smem, st, a);
    return cudaGetLastError();
}

// q's point sets were prepared (rows_prepare); a: the arguments of the
// chunk kernel, whose point pointers are replaced by the pair copies.
frnn_status enqueue_row_query(const QueryLaunch& q, const QueryArgs& a0, cudaStream_t st,
                              std::string& err) {
    const GridBufs& qs = *q.qset;
    const GridBufs& rs = *q.rset;
    if (!qs.rows_ready || !rs.rows_ready) {
        err = "row-task kernel launched without prepared inputs";
        return FRNN_ERR_INVALID_ARG;
    }
    QueryArgs a = a0;
    a.tasks = qs.row_tasks;
    a.ntasks = qs.scalars + kScNTasks;
    a.qpts = qs.ppts;
    a.rpts = rs.ppts;
    a.r2_screen = std::nextafter((float)((double)q.r2 * (1.0 + 0x1p-16)), INFINITY);
    cudaError_t ce = cudaSuccess;
    switch (rs.D) {
#define FRNN_CASE(d) case d: ce = launch_row_query_d<d>(a, q.exit_dims, q.num_sms, st); break;
        FRNN_CASE(1) FRNN_CASE(2) FRNN_CASE(3) FRNN_CASE(4) FRNN_CASE(5) FRNN_CASE(6)
        FRNN_CASE(7) FRNN_CASE(8) FRNN_CASE(9) FRNN_CASE(10) FRNN_CASE(11) FRNN_CASE(12)
        FRNN_CASE(13) FRNN_CASE(14) FRNN_CASE(15) FRNN_CASE(16)
#undef FRNN_CASE
        default:
            err = "unsupported D";
            return FRNN_ERR_INVALID_ARG;
    }
    if (ce != cudaSuccess) {
        err = std::string("row-task query launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    return FRNN_OK;
}

}  // namespace frnn
