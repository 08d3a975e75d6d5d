// query.cu — grid-path fixed-radius query: per-warp scan of the neighbouring
// cells with candidate tiles staged in shared memory by bulk copies, the exact
// float32 screen, and warp-level top-K.
//
// Method (Eq. 1, Sec. 1): for each query, every reference in the cells within
// +-m cells along each gridded axis is a candidate (complete by the grid's
// roundoff-safe construction, build.cu); each candidate's squared distance is
// computed under the fixed float32 contract and kept if <= fl(r*r).
//
// Organisation on the GPU (differs from the paper's thread-per-query kernel,
// whose profile showed dependent-load latency and divergence, Sec. 4.2):
//   * a persistent grid; each warp takes warp tasks (32 cell-sorted queries in
//     one row of cells) from an atomic counter;
//   * the candidates of a task are the union of its lanes' neighbourhoods: per
//     neighbour row one contiguous slot range; ranges are cut into tiles that
//     lane 0 copies into the warp's shared-memory ring with cp.async.bulk,
//     completion tracked by one mbarrier per buffer (prefetch depth kNBuf-1);
//   * every lane screens every candidate of the tile (broadcast shared loads):
//     warp-uniform control flow, no per-lane candidate lists;
//   * exact early rejection: after the first `EXIT` dimensions the warp votes;
//     partial sums never decrease (round-to-nearest of non-negative terms), so
//     if every lane's partial sum is already > r2 the candidate is rejected
//     for all of them without changing any verdict (the paper's "roundoff-safe
//     early rejection", Sec. 6).  Gridded axes are the last ones by default,
//     so the first dimensions are the ungridded, most selective ones;
//   * survivors are appended (d2, original index) straight into the query's
//     output row (the original index is looked up only for survivors: the
//     paper's deferred lookup, Table 3);
//   * at the end of the task the warp sorts each query's row by
//     (d2 bits << 32 | index) with a register bitonic network (shuffles) and
//     rewrites it coalesced with its padding.  Degree > K is rare (never in
//     the tracking-like workloads) and goes to an exact selection kernel.
#include <algorithm>

#include "frnn_host.h"

namespace frnn {

constexpr int kQueryWarps = 8;
constexpr int kNBuf = 3;
constexpr uint32_t kFull = 0xffffffffu;

template <int D>
struct QCfg {
    static constexpr int DP = padded_dim(D);
    // candidates per tile: about 2 KB per buffer
    static constexpr int TILE = DP == 4 ? 128 : (DP == 8 ? 64 : (DP == 12 ? 48 : 32));
    static constexpr int EXIT = D <= 4 ? D : 2;                         // default vote point
};

__host__ __device__ constexpr size_t query_smem_bytes(int DP, int TILE) {
    return (size_t)kQueryWarps * kNBuf * TILE * DP * sizeof(float) +
           (size_t)kQueryWarps * kNBuf * sizeof(uint64_t);
}

// ------------------------------------------------------------- top-K sorting

__device__ __forceinline__ uint64_t make_key(float d2, int32_t j) {
    return ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)j;
}

// Ascending bitonic sort of 32*R keys held by one warp: element e = i*32+lane
// lives in register v[i].
template <int R>
__device__ __forceinline__ void warp_bitonic(uint64_t (&v)[R]) {
    const int lane = threadIdx.x & 31;
    constexpr int N = 32 * R;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jr = j >> 5;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    if ((i & jr) == 0) {
                        const int e = i * 32 + lane;
                        const bool up = (e & k) == 0;
                        const uint64_t a = v[i], b = v[i | jr];
                        const bool sw = up ? (a > b) : (a < b);
                        v[i] = sw ? b : a;
                        v[i | jr] = sw ? a : b;
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int e = i * 32 + lane;
                    const uint64_t o = __shfl_xor_sync(kFull, v[i], j);
                    const bool lower = (lane & j) == 0;
                    const bool up = (e & k) == 0;
                    const bool keep_min = (lower == up);
                    const uint64_t mn = v[i] < o ? v[i] : o;
                    const uint64_t mx = v[i] < o ? o : v[i];
                    v[i] = keep_min ? mn : mx;
                }
            }
        }
    }
}

template <int R>
__device__ void sort_row_t(int32_t* irow, float* drow, int c, int K) {
    const int lane = threadIdx.x & 31;
    uint64_t v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int e = i * 32 + lane;
        v[i] = e < c ? make_key(drow[e], irow[e]) : ~0ull;
    }
    warp_bitonic<R>(v);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int e = i * 32 + lane;
        if (e < K) {
            const bool real = e < c;
            irow[e] = real ? (int32_t)(uint32_t)v[i] : -1;
            drow[e] = real ? __uint_as_float((uint32_t)(v[i] >> 32)) : INFINITY;
        }
    }
    for (int e = 32 * R + lane; e < K; e += 32) {
        irow[e] = -1;
        drow[e] = INFINITY;
    }
}

// Rows longer than this (or with degree > K) are finished by the selection
// kernel below, which keeps the register footprint of the scan kernel small.
constexpr int kFastSortMax = 128;

// Sort the first c (<= min(K, kFastSortMax)) entries of a row in place and pad
// the rest.
__device__ __noinline__ void finalize_row(int32_t* irow, float* drow, int c, int K) {
    const int lane = threadIdx.x & 31;
    if (c <= 1) {
        for (int e = c + lane; e < K; e += 32) {
            irow[e] = -1;
            drow[e] = INFINITY;
        }
        return;
    }
    if (c <= 32) sort_row_t<1>(irow, drow, c, K);
    else if (c <= 64) sort_row_t<2>(irow, drow, c, K);
    else sort_row_t<4>(irow, drow, c, K);
}

// ------------------------------------------------------------- grid query

struct TaskGeom {
    int total_tiles;
    int rs, re, tp;   // this lane's neighbour-row slot range and inclusive tile prefix
};

template <int TILE>
__device__ __forceinline__ void tile_info(const TaskGeom& g, int t, int& base, int& len) {
    const unsigned below = __ballot_sync(kFull, g.tp <= t);
    const int L = __popc(below);
    const int rs = __shfl_sync(kFull, g.rs, L);
    const int re = __shfl_sync(kFull, g.re, L);
    const int tp = __shfl_sync(kFull, g.tp, L);
    const int ntl = (re - rs + TILE - 1) / TILE;
    const int first = tp - ntl;
    base = rs + (t - first) * TILE;
    len = min(TILE, re - base);
}

template <int D, int EXIT>
__global__ void __launch_bounds__(kQueryWarps * 32, 3) k_grid_query(QueryArgs a) {
    using C = QCfg<D>;
    constexpr int DP = C::DP;
    constexpr int TILE = C::TILE;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* ring = reinterpret_cast<float*>(smem) + (size_t)warp * kNBuf * TILE * DP;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)kQueryWarps * kNBuf * TILE * DP *
                                                            sizeof(float)) +
                     warp * kNBuf;
    if (lane == 0)
        for (int b = 0; b < kNBuf; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
    __syncwarp();
    uint32_t phase = 0;   // bit b: parity to wait for on buffer b

    const int ntasks = *a.ntasks;
    const float r2 = a.r2;
    const int K = a.K;

    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.task_counter, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= ntasks) break;
        const Task task = a.tasks[t];
        const EventHdr& h = a.ev[task.ev];
        int32_t* counts = a.counts ? a.counts : h.counts;
        int32_t* oidx = a.counts ? a.idx : h.idx;
        float* od2 = a.counts ? a.dist2 : h.dist2;

        const bool act = lane < task.nq;
        const int qs = task.qslot + lane;
        const int qorig = act ? a.qperm[qs] : 0;
        if (!h.valid) {
            // grid built from non-finite input: empty rows (frnn_sync reports it)
            for (int ql = 0; ql < task.nq; ++ql) {
                const int qo = __shfl_sync(kFull, qorig, ql);
                finalize_row(oidx + (int64_t)qo * K, od2 + (int64_t)qo * K, 0, K);
                if (lane == 0) counts[qo] = 0;
            }
            continue;
        }
        float q[DP];
        if (act) {
            const float4* src = reinterpret_cast<const float4*>(a.qpts + (int64_t)qs * DP);
#pragma unroll
            for (int k4 = 0; k4 < DP / 4; ++k4) {
                float4 v = src[k4];
                q[4 * k4 + 0] = v.x; q[4 * k4 + 1] = v.y; q[4 * k4 + 2] = v.z; q[4 * k4 + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < DP; ++k) q[k] = __int_as_float(0x7fc00000);   // NaN: never accepted
        }
        const int qc = act ? a.qcell[qs] : 0;
        const int dims0 = h.dims[0], dims1 = h.dims[1], dims2 = h.dims[2], m = h.m;
        const int x = qc % dims0;
        const int xa = __shfl_sync(kFull, x, 0);
        const int xb = __shfl_sync(kFull, x, task.nq - 1);
        const int y = task.row % dims1, z = task.row / dims1;
        const int side = 2 * m + 1;
        const int nrows = h.naxes >= 3 ? side * side : (h.naxes == 2 ? side : 1);

        TaskGeom g;
        g.rs = 0;
        g.re = 0;
        if (lane < nrows) {
            const int dy = h.naxes >= 2 ? (lane % side) - m : 0;
            const int dz = h.naxes >= 3 ? (lane / side) - m : 0;
            const int yy = y + dy, zz = z + dz;
            if (yy >= 0 && yy < dims1 && zz >= 0 && zz < dims2) {
                const int64_t rowbase = h.cell_off + (int64_t)(yy + dims1 * zz) * dims0;
                const int x0 = max(xa - m, 0), x1 = min(xb + m, dims0 - 1);
                g.rs = a.cstart[rowbase + x0];
                g.re = a.cstart[rowbase + x1 + 1];
            }
        }
        const int ntl = (g.re - g.rs + TILE - 1) / TILE;
        int tp = ntl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, tp, o);
            if (lane >= o) tp += v;
        }
        g.tp = tp;
        g.total_tiles = __shfl_sync(kFull, tp, 31);

        int32_t* irow = oidx + (int64_t)qorig * K;
        float* drow = od2 + (int64_t)qorig * K;
        int cnt = 0;
        const int self_slot = a.self ? qs : -1;

        // prologue: fill the ring
        const int pre = min(kNBuf, g.total_tiles);
        for (int tt = 0; tt < pre; ++tt) {
            int base, len;
            tile_info<TILE>(g, tt, base, len);
            if (lane == 0) {
                const uint32_t bytes = (uint32_t)len * DP * sizeof(float);
                mbar_arrive_expect_tx(&bars[tt], bytes);
                bulk_g2s(ring + (size_t)tt * TILE * DP, a.rpts + (int64_t)base * DP, bytes,
                         &bars[tt]);
            }
        }
        int timed_out_at = -1;
        for (int tt = 0; tt < g.total_tiles; ++tt) {
            const int b = tt % kNBuf;
            int base, len;
            tile_info<TILE>(g, tt, base, len);
            if (!mbar_wait_bounded(&bars[b], (phase >> b) & 1u)) {
                timed_out_at = tt;
                break;
            }
            phase ^= 1u << b;
            const float* tile = ring + (size_t)b * TILE * DP;
#pragma unroll 2
            for (int c = 0; c < len; ++c) {
                const float4* cp4 = reinterpret_cast<const float4*>(tile + c * DP);
                float cv[DP];
#pragma unroll
                for (int k4 = 0; k4 < DP / 4; ++k4) {
                    float4 v = cp4[k4];
                    cv[4 * k4 + 0] = v.x; cv[4 * k4 + 1] = v.y;
                    cv[4 * k4 + 2] = v.z; cv[4 * k4 + 3] = v.w;
                }
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < EXIT; ++k) {
                    const float d = __fsub_rn(q[k], cv[k]);
                    s = __fadd_rn(s, __fmul_rn(d, d));
                }
                if (EXIT < D) {
                    if (!__any_sync(kFull, s <= r2)) continue;
#pragma unroll
                    for (int k = EXIT; k < D; ++k) {
                        const float d = __fsub_rn(q[k], cv[k]);
                        s = __fadd_rn(s, __fmul_rn(d, d));
                    }
                }
                if (s <= r2) {
                    const int cs = base + c;
                    if (cs != self_slot) {
                        const int pos = cnt++;
                        if (pos < K) {
                            irow[pos] = a.rperm[cs];
                            drow[pos] = s;
                        }
                    }
                }
            }
            __syncwarp();
            const int nt = tt + kNBuf;
            if (nt < g.total_tiles) {
                int nbase, nlen;
                tile_info<TILE>(g, nt, nbase, nlen);
                if (lane == 0) {
                    fence_proxy_async_smem();
                    const uint32_t bytes = (uint32_t)nlen * DP * sizeof(float);
                    mbar_arrive_expect_tx(&bars[b], bytes);
                    bulk_g2s(ring + (size_t)b * TILE * DP, a.rpts + (int64_t)nbase * DP, bytes,
                             &bars[b]);
                }
            }
        }
        if (timed_out_at >= 0) {
            // record, wait (bounded) for the copies still in flight, stop this warp
            if (lane == 0) atomicOr(a.status, kStatusTimeout);
            const int issued = min(g.total_tiles, timed_out_at + kNBuf);
            for (int t2 = timed_out_at; t2 < issued; ++t2) {
                const int b2 = t2 % kNBuf;
                mbar_wait_bounded(&bars[b2], (phase >> b2) & 1u);
                phase ^= 1u << b2;
            }
            return;
        }
        __syncwarp();
        for (int ql = 0; ql < task.nq; ++ql) {
            const int c = __shfl_sync(kFull, cnt, ql);
            const int qo = __shfl_sync(kFull, qorig, ql);
            if (c > K || c > kFastSortMax) {
                if (lane == 0) {
                    const int pos = atomicAdd(a.ovf_count, 1);
                    if (pos < a.ovf_cap) {
                        a.ovf[pos].qslot = task.qslot + ql;
                        a.ovf[pos].ev = task.ev;
                    } else {
                        atomicOr(a.status, kStatusCapacity);
                    }
                }
                continue;
            }
            finalize_row(oidx + (int64_t)qo * K, od2 + (int64_t)qo * K, c, K);
            if (lane == 0) counts[qo] = c;
        }
    }
}

// ------------------------------------------------------------- overflow path
// Exact selection for queries whose degree exceeds K (or whose row is longer
// than kFastSortMax, which needs K > 128): one warp per query scans
// the query's own +-m neighbourhood with lanes over candidates, appends keys
// below the current threshold to a shared buffer, and whenever the buffer is
// nearly full sorts it and keeps the K smallest (the threshold becomes the
// K-th key).  Keys are unique (indices differ), so the K smallest are unique.

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
        const float* qp = a.qpts + (int64_t)qs * DP;
        const int qc = a.qcell[qs];
        const int dims0 = h.dims[0], dims1 = h.dims[1], dims2 = h.dims[2], m = h.m;
        const int x = qc % dims0, y = (qc / dims0) % dims1, z = qc / (dims0 * dims1);
        const int self_slot = a.self ? qs : -1;
        int fill = 0;
        int64_t deg = 0;
        uint64_t thr = ~0ull;
        for (int i = lane; i < cap; i += 32) buf[i] = ~0ull;
        __syncwarp();
        const int ylo = h.naxes >= 2 ? max(y - m, 0) : 0, yhi = h.naxes >= 2 ? min(y + m, dims1 - 1) : 0;
        const int zlo = h.naxes >= 3 ? max(z - m, 0) : 0, zhi = h.naxes >= 3 ? min(z + m, dims2 - 1) : 0;
        for (int zz = zlo; zz <= zhi; ++zz) {
            for (int yy = ylo; yy <= yhi; ++yy) {
                const int64_t rowbase = h.cell_off + (int64_t)(yy + dims1 * zz) * dims0;
                const int rs = a.cstart[rowbase + max(x - m, 0)];
                const int re = a.cstart[rowbase + min(x + m, dims0 - 1) + 1];
                for (int c0 = rs; c0 < re; c0 += 32) {
                    const int cs = c0 + lane;
                    uint64_t key = ~0ull;
                    if (cs < re && cs != self_slot) {
                        const float* cp = a.rpts + (int64_t)cs * DP;
                        float s = 0.f;
                        for (int k = 0; k < D; ++k) {
                            const float d = __fsub_rn(qp[k], cp[k]);
                            s = __fadd_rn(s, __fmul_rn(d, d));
                        }
                        if (s <= a.r2) {
                            key = make_key(s, a.rperm[cs]);
                            ++deg;
                            if (key >= thr) key = ~0ull;
                        }
                    }
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
        smem_bitonic(buf, cap);
        int32_t* irow = oidx + (int64_t)qo * K;
        float* drow = od2 + (int64_t)qo * K;
        for (int e = lane; e < K; e += 32) {
            const uint64_t v = buf[e];
            const bool real = v != ~0ull;
            irow[e] = real ? (int32_t)(uint32_t)v : -1;
            drow[e] = real ? __uint_as_float((uint32_t)(v >> 32)) : INFINITY;
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) deg += __shfl_xor_sync(kFull, deg, o2);
        if (lane == 0) (a.counts ? a.counts : h.counts)[qo] = (int32_t)(deg < K ? deg : K);
        __syncwarp();
    }
}

// ------------------------------------------------------------- host launch

template <int D>
static cudaError_t launch_grid_query_d(const QueryArgs& a, int exit_dims, int num_sms,
                                       cudaStream_t st) {
    using C = QCfg<D>;
    const size_t smem = query_smem_bytes(C::DP, C::TILE);
    auto kern = &k_grid_query<D, C::EXIT>;
    // other vote points are compiled for the tracking-like dimensions only
    if constexpr (D == 8 || D == 12) {
        if (exit_dims == 1) kern = &k_grid_query<D, 1>;
        else if (exit_dims == 3) kern = &k_grid_query<D, 3>;
        else if (exit_dims == 4) kern = &k_grid_query<D, 4>;
        else if (exit_dims >= 5) kern = &k_grid_query<D, 6>;
    }
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (ce != cudaSuccess) return ce;
    int per_sm = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kQueryWarps * 32, smem);
    if (ce != cudaSuccess) return ce;
    per_sm = std::max(per_sm, 1);
    kern<<<num_sms * per_sm, kQueryWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

frnn_status enqueue_grid_query(const QueryLaunch& q, cudaStream_t st, std::string& err) {
    const GridBufs& qs = *q.qset;
    const GridBufs& rs = *q.rset;
    QueryArgs a{};
    a.ev = rs.hdr;
    a.tasks = qs.tasks;
    a.ntasks = qs.scalars + kScNTasks;
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
    a.exit_dims = q.exit_dims;
    cudaMemsetAsync(qs.scalars + kScTaskCounter, 0, 2 * sizeof(int32_t), st);   // counter + ovf
    cudaError_t ce = cudaSuccess;
    switch (rs.D) {
#define FRNN_CASE(d) case d: ce = launch_grid_query_d<d>(a, q.exit_dims, q.num_sms, st); break;
        FRNN_CASE(1) FRNN_CASE(2) FRNN_CASE(3) FRNN_CASE(4) FRNN_CASE(5) FRNN_CASE(6)
        FRNN_CASE(7) FRNN_CASE(8) FRNN_CASE(9) FRNN_CASE(10) FRNN_CASE(11) FRNN_CASE(12)
        FRNN_CASE(13) FRNN_CASE(14) FRNN_CASE(15) FRNN_CASE(16)
#undef FRNN_CASE
        default:
            err = "unsupported D";
            return FRNN_ERR_INVALID_ARG;
    }
    if (ce != cudaSuccess) {
        err = std::string("grid query launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    // overflow pass: buffer of a power of two >= 2K keys per warp
    int cap = 64;
    while (cap < 2 * q.K) cap <<= 1;
    const size_t osmem = (size_t)kOvfWarps * cap * sizeof(uint64_t);
    ce = cudaFuncSetAttribute(k_overflow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osmem);
    if (ce == cudaSuccess) {
        k_overflow<<<q.num_sms, kOvfWarps * 32, osmem, st>>>(a, cap);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) {
        err = std::string("overflow launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    return FRNN_OK;
}

}  // namespace frnn
