// build.cu — uniform-grid build: bounding boxes, cell parameters, cell ids,
// counting sort into cell-sorted padded rows, and the warp-task list.
//
// The uniform grid / cell list is the method of the original FRNN the paper
// starts from (Sec. 2: uniform-grid kernel, spacing chosen so that r is an
// integer multiple of it).  Here at most 5 coordinates are gridded; the cell
// assignment is "roundoff-safe" (Table 1): it provably never separates two
// points the float32 contract accepts by more than m cells per axis (proof at
// event_params below).
//
// Steps, all on the device, no host synchronisation:
//   k_init      zero the cell counts, reset bounding boxes (and, for one event,
//               write the per-event tables passed by value)
//   k_bbox      per-event per-axis min / max (+ non-finite flag), float4 staged;
//               the event's last block to finish derives the grid parameters:
//               gridded axes, cell edge, cells per axis
//   k_cellid    cell id of every point and its rank inside the cell (atomics)
//   scan        exclusive warp-shuffle prefix scan of the counts -> cell starts
//   k_scatter   slot -> original index, slot -> cell, and the point's row of
//               DP floats at its slot (cell-sorted coordinates)
// (the tensor-core path adds its 128-query tiles: k_rowtasks, a scan, k_emit)
#include <algorithm>
#include <cmath>

#include "frnn_host.h"

namespace frnn {

// ------------------------------------------------------------------ helpers

// Entry of each event's box copy 0 that counts its finished k_bbox blocks.
constexpr int kBBoxDone = 33;
static_assert(kBBoxDone >= 33 && kBBoxDone < kBBoxStride, "after the minima, maxima and flag");

// The tables of a one-event build (header, block starts, cell offsets), passed
// to k_init by value instead of being copied from the host.
struct OneEventTables {
    EventHdr hdr;
    int64_t cell_end;   // cell_off[1]
    int32_t nblk;       // blk_start[1]
    int32_t set;        // 0: the tables are already on the device
};

// A one-event build's input, passed by value to the kernels that stage it:
// they stage their block's points before waiting for the previous kernel of
// the chain (no kernel of the chain writes the caller's points, and the
// header that would locate them is written by k_init in this case).
struct EarlyPts {
    const float* refs;
    int64_t n;
    int32_t set;   // 0: locate the points through the tables, after the wait
};

// Stage this block's input rows before the wait when the build is one event.
__device__ __forceinline__ bool stage_early(float* sm, const EarlyPts& ep, int D, bool pad);

__device__ __forceinline__ int find_event(const int32_t* starts, int E, int b) {
    // largest e with starts[e] <= b
    int lo = 0, hi = E - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_event64(const int64_t* starts, int E, int64_t i) {
    int lo = 0, hi = E - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Staged point rows in shared memory: float j of the block's rows sits at
// j + j / 32 when D is a multiple of 4 (one padding word per 32), else at j,
// so that a warp reading coordinate k of 32 consecutive rows (stride D) hits
// distinct banks for D = 4, 8, 16 and at most two per bank otherwise.
__device__ __forceinline__ int stage_slot(int j, bool pad) { return pad ? j + (j >> 5) : j; }
__host__ __device__ constexpr size_t staged_floats(int D) {
    return (size_t)kBuildPtsPerBlock * D + (size_t)kBuildPtsPerBlock * D / 32 + 1;
}

// Row i of the staged rows, indexed by coordinate.
struct StagedRow {
    const float* sm;
    int j0;
    bool pad;
    __device__ __forceinline__ float operator[](int k) const { return sm[stage_slot(j0 + k, pad)]; }
};

// Stage nf consecutive floats of a row-major point array into shared memory
// (at stage_slot), using 16-byte vector loads for the aligned body.
__device__ __forceinline__ void stage_floats(float* sm, const float* src, int nf, bool pad) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    int head = (int)(((16u - (uint32_t)(a & 15u)) & 15u) >> 2);
    if (a & 3u) head = nf;   // not even 4-byte aligned: scalar path (cannot happen for float*)
    head = min(head, nf);
    for (int i = threadIdx.x; i < head; i += blockDim.x) sm[stage_slot(i, pad)] = __ldg(src + i);
    const int n4 = (nf - head) >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(src + head);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        float4 v = __ldg(s4 + i);
        const int j = head + 4 * i;
        sm[stage_slot(j, pad)] = v.x;
        sm[stage_slot(j + 1, pad)] = v.y;
        sm[stage_slot(j + 2, pad)] = v.z;
        sm[stage_slot(j + 3, pad)] = v.w;
    }
    for (int i = head + 4 * n4 + threadIdx.x; i < nf; i += blockDim.x)
        sm[stage_slot(i, pad)] = __ldg(src + i);
}

__device__ __forceinline__ bool stage_early(float* sm, const EarlyPts& ep, int D, bool pad) {
    if (!ep.set) return false;
    const int64_t p0 = (int64_t)blockIdx.x * kBuildPtsPerBlock;
    const int np = (int)min((int64_t)kBuildPtsPerBlock, ep.n - p0);
    if (np > 0) stage_floats(sm, ep.refs + p0 * D, np * D, pad);
    return true;
}

// Cell coordinate along one gridded axis: floor(fl(fl(x' - lo) * inv_h))
// clamped to [0, dim - 1], with x' = x clamped to [lo, hi].  Every kernel that
// bins points (references and queries) uses exactly this function.
__device__ __forceinline__ int cell_coord(float x, float lo, float hi, float inv_h, int dim) {
    float xc = fminf(fmaxf(x, lo), hi);
    float g = __fmul_rn(__fsub_rn(xc, lo), inv_h);
    int c = __float2int_rd(g);
    return min(max(c, 0), dim - 1);
}

template <class Row>
__device__ __forceinline__ int point_cell(const Row& p, const EventHdr& h) {
    int c = 0, stride = 1;
#pragma unroll
    for (int a = 0; a < kMaxAxes; ++a) {
        if (a < h.naxes) {
            c += cell_coord(p[h.axes[a]], h.lo[a], h.hi[a], h.inv_h, h.dims[a]) * stride;
            stride *= h.dims[a];
        }
    }
    return c;
}

// ------------------------------------------------------------------ kernels

__global__ void k_init(int32_t* counts, int64_t L, int32_t* bbox, int E, int32_t* scalars,
                       int32_t bb_min_init, int32_t bb_max_init, OneEventTables t1,
                       EventHdr* hdr, int32_t* blk_start, int64_t* cell_off) {
    pdl_trigger();
    pdl_wait();   // the previous work on the stream may still read the tables
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t1.set && i == 0) {
        hdr[0] = t1.hdr;
        blk_start[0] = 0;
        blk_start[1] = t1.nblk;
        cell_off[0] = 0;
        cell_off[1] = t1.cell_end;
    }
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // counts: 16-byte stores (the array starts 256-byte aligned)
    int4* c4 = reinterpret_cast<int4*>(counts);
    const int64_t L4 = L / 4;
    for (int64_t j = i; j < L4; j += stride) c4[j] = make_int4(0, 0, 0, 0);
    for (int64_t j = 4 * L4 + i; j < L; j += stride) counts[j] = 0;
    for (int64_t j = i; j < (int64_t)E * kBBoxCopies * kBBoxStride; j += stride) {
        int k = (int)(j % kBBoxStride);
        bbox[j] = k < 16 ? bb_min_init : (k < 32 ? bb_max_init : 0);   // flag, block counter: 0
    }
    if (i < kScalars) scalars[i] = 0;
}

__device__ void event_params(EventHdr* hdr, int e, int D, const int32_t* bbox, float r, int m,
                             int axes_mode, int naxes_req, int32_t* counts);

// Per-event bounding boxes.  One CTA per build block (256 points staged
// through shared memory with 16-byte loads) reduces its points and merges the
// result into one of kBBoxCopies copies of the event's box (copy = block mod
// kBBoxCopies), so that no address takes more than a few dozen atomics.  The
// event's last block to finish (a counter beside copy 0, taken after a memory
// fence) combines the copies and derives the grid parameters.
// (at most 40 registers, as without the parameter step: six CTAs per SM; the
// one-thread parameter code may spill)
__global__ void __launch_bounds__(kBuildPtsPerBlock, 6) k_bbox(EventHdr* hdr,
                                                            const int32_t* blk_start, int E,
                                                            int D, int32_t* bbox,
                                                            int32_t* status, float r, int m,
                                                            int axes_mode, int naxes_req,
                                                            int32_t* counts, EarlyPts ep) {
    pdl_trigger();
    extern __shared__ float sm[];
    const bool pad = (D & 3) == 0;
    const bool staged = stage_early(sm, ep, D, pad);
    pdl_wait();
    __shared__ float red_mn[kMaxD][kBuildPtsPerBlock / 32];
    __shared__ float red_mx[kMaxD][kBuildPtsPerBlock / 32];
    __shared__ int red_bad;
    const int e = find_event(blk_start, E, blockIdx.x);
    const EventHdr& h = hdr[e];
    const int64_t p0 = (int64_t)(blockIdx.x - blk_start[e]) * kBuildPtsPerBlock;
    const int np = (int)min((int64_t)kBuildPtsPerBlock, h.n - p0);
    if (threadIdx.x == 0) red_bad = 0;
    if (!staged && np > 0) stage_floats(sm, h.refs + p0 * D, np * D, pad);
    __syncthreads();
    float mn[kMaxD], mx[kMaxD];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < kMaxD; ++k) { mn[k] = INFINITY; mx[k] = -INFINITY; }
    if ((int)threadIdx.x < np) {
        const StagedRow p{sm, (int)threadIdx.x * D, pad};
#pragma unroll
        for (int k = 0; k < kMaxD; ++k) {
            if (k < D) {
                float v = p[k];
                bad |= !isfinite(v);
                mn[k] = fminf(mn[k], v);
                mx[k] = fmaxf(mx[k], v);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kMaxD; ++k) {
        if (k < D) {
            float a = mn[k], b = mx[k];
            for (int o = 16; o > 0; o >>= 1) {
                a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
                b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
            }
            if (lane == 0) { red_mn[k][warp] = a; red_mx[k][warp] = b; }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&red_bad, 1);
    __syncthreads();
    int32_t* bb = bbox + ((int64_t)e * kBBoxCopies + (blockIdx.x % kBBoxCopies)) * kBBoxStride;
    if (threadIdx.x < (unsigned)D) {
        const int k = threadIdx.x;
        float a = INFINITY, b = -INFINITY;
        for (int w = 0; w < kBuildPtsPerBlock / 32; ++w) {
            a = fminf(a, red_mn[k][w]);
            b = fmaxf(b, red_mx[k][w]);
        }
        atomicMin(bb + k, float_to_ordered(a));
        atomicMax(bb + 16 + k, float_to_ordered(b));
    }
    if (threadIdx.x == 0 && red_bad) {
        atomicOr(bb + 32, 1);
        atomicOr(status, kStatusNonFinite);
    }
    __shared__ int s_last;
    __threadfence();   // this block's box updates before its count
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nb = blk_start[e + 1] - blk_start[e];
        int32_t* done = bbox + (int64_t)e * kBBoxCopies * kBBoxStride + kBBoxDone;
        s_last = atomicAdd(done, 1) == nb - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();   // every other block's updates before the reads
    event_params(hdr, e, D, bbox, r, m, axes_mode, naxes_req, counts);
}

// Grid parameters of one event (one CTA: its warps combine the box copies,
// then warp 0 derives the parameters, lane a handling gridded axis a).
//
// Roundoff-safe cell assignment (proof).  Let u = 2^-24.  If the contract
// accepts (x, y), every rounded square t_a = fl(fl(x_a - y_a)^2) is <= the
// final sum s (partial sums of non-negative terms never decrease under
// round-to-nearest) and s <= r2 = fl(r*r) <= r^2 (1 + u); with r2 normal this
// gives |fl(x_a - y_a)| <= r (1 + 2u) and |x_a - y_a| <= rho := r (1 + 2^-20).
// For lo <= x <= y <= hi the cell coordinate g(.) = fl(fl(. - lo) * inv_h) is
// monotone and g(y) - g(x) <= inv_h (rho + 2^-21 E) + 2^-148, E = hi - lo.  If
// that bound is < m, floor(g(y)) - floor(g(x)) <= m, and clamping to
// [0, dim-1] keeps it so; queries are clamped to [lo, hi] first, which only
// shrinks their distance to any reference.  So searching +-m cells per gridded
// axis finds every accepted pair.  The bound is evaluated in float32 with
// every operation rounded upward (rho, E and each step), which can only
// overestimate it: inv_h starts at fl_down(m / fl_up(r (1+2^-10))) and is
// lowered until the overestimate is below m - 2^-20, every axis has at most
// 1024 cells and the event's cell count fits its capacity.
static_assert(kBBoxCopies == 32, "one copy per lane when the copies are combined");

static_assert(kBuildPtsPerBlock == 256, "eight warps combine the box copies");
static_assert(kMaxD <= 32 && kMaxAxes <= 32, "one lane per coordinate");

// One candidate grid, held by warp 0: k gridded axes (the last k coordinates,
// or the k widest), cell multiple m, the cell edge fitted to the proof's
// condition, 1024 cells per axis and the event's cell budget, and the
// expected fraction of the event a query's neighbourhood covers if the
// points were spread evenly: the product over the gridded axes of
// min(1, (2m+1) cells / extent).  The parameter step keeps the candidate
// with the smallest fraction; the choice never changes results.  Lane a < k
// holds gridded axis a (coordinate, cells, extremes); the other fields are
// the same on every lane.
struct GridFit {
    int naxes = 1, m = 1;
    int axis = 0, dim = 1;
    float lo = 0.f, hi = 0.f;
    float inv_h = 0.f;
    int32_t ncells = 1;
    float frac = INFINITY;
    bool at_start = false;   // the starting cell edge fitted (no enlargement)
};

// lo_j, hi_j: the extremes of coordinate j on lane j < D.  Called by all
// lanes of warp 0.
__device__ void grid_fit(GridFit& f, float lo_j, float hi_j, int D, int k, int m, int axes_mode,
                         float r, int64_t cap, bool valid, int max_rows) {
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    f.naxes = k;
    // neighbour rows, (2m+1)^(k-1): at most max_rows (the chunk kernel
    // enumerates kMaxNbrRows, 32 per round; the row-task kernel one per lane)
    int mm = max(m, 1);
    for (;;) {
        int rows = 1;
        for (int a = 1; a < k; ++a) rows *= 2 * mm + 1;
        if (rows <= max_rows || mm == 1) break;
        --mm;
    }
    f.m = mm;
    int ax = lane < k ? D - k + lane : 0;
    if (valid && axes_mode == 1 && D > k) {
        // the k widest coordinates (ties by lower index), in index order
        const float wj = __fsub_rn(hi_j, lo_j);
        int rank = 0;
        for (int i = 0; i < D; ++i) {
            const float wi = __shfl_sync(kAll, wj, i);
            if (wi > wj || (wi == wj && i < lane)) ++rank;
        }
        const unsigned sel = __ballot_sync(kAll, lane < D && rank < k);
        int cnt = 0;
        ax = 0;
        for (int j = 0; j < D; ++j) {
            if ((sel >> j) & 1u) {
                if (cnt == lane) ax = j;
                ++cnt;
            }
        }
    }
    const float lo = __shfl_sync(kAll, lo_j, ax);
    const float hi = __shfl_sync(kAll, hi_j, ax);
    f.axis = lane < k ? ax : 0;
    f.lo = lo;
    f.hi = hi;
    if (!valid) {
        f.frac = 1.f;
        return;
    }
    // the cell coordinate of hi is floor(fl(ext * inv_h)): dim = that + 1
    const float ext = __fsub_rn(hi, lo);
    const float ext_up = __fsub_ru(hi, lo);
    const float rho_up = __fmul_ru(r, 1.0f + 0x1p-20f);
    const float need = (float)mm - 0x1p-20f;
    float ih = __fdiv_rd((float)mm, __fmul_ru(r, 1.0f + 0x1p-10f));
    int dim = 1;
    int64_t cells = 1;
    bool fit = false;
    for (int it = 0; it < 4096; ++it) {
        bool ok = true;
        dim = 1;
        if (lane < k) {
            const float c = floorf(__fmul_rn(ext, ih)) + 1.0f;
            if (!(c <= (float)kMaxDimsPerAxis)) ok = false;
            else dim = (int)c;
            const float bound =
                __fadd_ru(__fmul_ru(ih, __fadd_ru(rho_up, __fmul_ru(0x1p-21f, ext_up))), 0x1p-148f);
            if (!(bound < need)) ok = false;
        }
        cells = 1;
        for (int a = 0; a < k; ++a) cells *= __shfl_sync(kAll, dim, a);
        if (__all_sync(kAll, ok) && cells <= cap) {
            fit = true;
            f.at_start = it == 0;
            break;
        }
        ih = __fmul_rd(ih, 0.9f);
        if (!(ih > 0.f)) break;
    }
    if (!fit) {   // one cell is always safe
        ih = 0.f;
        dim = 1;
        cells = 1;
    }
    f.dim = lane < k ? dim : 1;
    f.inv_h = ih;
    f.ncells = (int32_t)cells;
    float fr = 1.f;
    if (lane < k && ext_up > 0.f) {
        const float span = ih > 0.f ? (2.f * (float)mm + 1.f) / ih : INFINITY;
        fr = fminf(1.f, span / ext_up);
    }
    float frac = 1.f;
    for (int a = 0; a < k; ++a) frac *= __shfl_sync(kAll, fr, a);
    f.frac = frac;
}

__device__ void event_params(EventHdr* hdr, int e, int D, const int32_t* bbox, float r, int m,
                             int axes_mode, int naxes_req, int32_t* counts) {
    __shared__ int32_t bb[kBBoxStride];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // lane c holds copy c of entry k; a warp reduction combines them (all of a
    // warp's loads are issued before the first reduction)
    constexpr int kPer = (kBBoxStride + 7) / 8;
    int32_t v[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int k = warp + 8 * i;
        // L2 reads: the copies were updated by other blocks' atomics
        v[i] = k < kBBoxStride ? __ldcg(bbox + ((int64_t)e * kBBoxCopies + lane) * kBBoxStride + k) : 0;
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int k = warp + 8 * i;
        for (int o = 16; o > 0; o >>= 1) {
            const int32_t x = __shfl_xor_sync(0xffffffffu, v[i], o);
            v[i] = k < 16 ? min(v[i], x) : (k < 32 ? max(v[i], x) : (v[i] | x));
        }
        if (lane == 0 && k < kBBoxStride) bb[k] = v[i];
    }
    __syncthreads();
    if (warp != 0) return;
    EventHdr& H = hdr[e];
    const int64_t n = H.n;
    const int64_t cell_off = H.cell_off;
    const int32_t cell_cap = H.cell_cap;
    // per-event presets (batched autotuning) win over the call's options;
    // 0 = automatic: the widest count up to kMaxAxes, or one fewer axis when
    // the cell budget makes that grid's neighbourhoods smaller
    const int want = H.naxes > 0 ? H.naxes : naxes_req;
    const int m_req = H.m > 0 ? H.m : m;
    __syncwarp();   // every lane has read the header before it is written
    // the last cell-array entry of the event counts its pair padding slot, so
    // the next event's slots start on a pair boundary
    if (lane == 0) counts[cell_off + cell_cap] = (int32_t)(n & 1);
    const float lo_j = lane < D ? ordered_to_float(bb[lane]) : 0.f;
    const float hi_j = lane < D ? ordered_to_float(bb[16 + lane]) : 0.f;
    const bool fin = lane >= D || (isfinite(lo_j) && isfinite(hi_j));
    const bool valid = __all_sync(0xffffffffu, fin) && bb[32] == 0 && n > 0;
    const int kmax = min(D, kMaxAxes);
    const int k_hi = want > 0 ? min(D, min(want, kMaxAxes)) : kmax;
    const int k_lo = want > 0 ? k_hi : max(1, kmax - 1);
    // grids requested with up to four axes are scanned by the row-task
    // kernel, whose lanes hold one neighbour row each
    const int max_rows = (want >= 1 && want <= 4) ? 32 : kMaxNbrRows;
    GridFit best;
    best.frac = INFINITY;
    for (int k = k_hi; k >= k_lo; --k) {
        GridFit f;
        grid_fit(f, lo_j, hi_j, D, k, m_req, axes_mode, r, cell_cap, valid, max_rows);
        if (f.frac < best.frac) best = f;
        // at the starting cell edge a grid over more axes covers at most the
        // fraction of one over fewer (one factor <= 1 more): no need to try fewer
        if (f.at_start) break;
    }
    const int na = best.naxes;
    if (lane < kMaxAxes) {
        const bool gridded = lane < na;
        H.axes[lane] = gridded ? best.axis : 0;
        H.dims[lane] = gridded && valid ? best.dim : 1;
        H.lo[lane] = gridded && valid ? best.lo : 0.f;
        H.hi[lane] = gridded && valid ? best.hi : 0.f;
    }
    if (lane < kMaxD) {
        float c = 0.f;
        if (valid && lane < D) {
            c = __fadd_rn(lo_j, __fmul_rn(0.5f, __fsub_rn(hi_j, lo_j)));
            if (!isfinite(c)) c = 0.f;
        }
        H.ctr[lane] = c;
    }
    if (lane == 0) {
        H.naxes = na;
        H.m = best.m;
        H.valid = valid ? 1 : 0;
        H.inv_h = valid ? best.inv_h : 0.f;
        H.ncells = valid ? best.ncells : 1;
    }
}

// Cross-set binning: take the reference grid's parameters for each event.
__global__ void k_copy_params(EventHdr* dst, const EventHdr* src, int E, int32_t* counts) {
    pdl_trigger();
    pdl_wait();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    EventHdr& d = dst[e];
    counts[d.cell_off + d.cell_cap] = (int32_t)(d.n & 1);
    const EventHdr& s = src[e];
    d.naxes = s.naxes;
    d.m = s.m;
    d.valid = s.valid;
    d.inv_h = s.inv_h;
    d.ncells = s.ncells;
    for (int a = 0; a < kMaxAxes; ++a) {
        d.axes[a] = s.axes[a];
        d.dims[a] = s.dims[a];
        d.lo[a] = s.lo[a];
        d.hi[a] = s.hi[a];
    }
    for (int k = 0; k < kMaxD; ++k) d.ctr[k] = s.ctr[k];
}

// Non-finite check of a query set binned with foreign parameters (the bbox
// kernel does it for reference sets).
__global__ void __launch_bounds__(kBuildPtsPerBlock) k_cellid(const EventHdr* hdr,
                                                              const int32_t* blk_start, int E,
                                                              int D, int32_t* counts,
                                                              int32_t* cid, int32_t* rnk,
                                                              int check_finite, int32_t* status,
                                                              EarlyPts ep) {
    pdl_trigger();
    extern __shared__ float sm[];
    const bool pad = (D & 3) == 0;
    const bool staged = stage_early(sm, ep, D, pad);
    pdl_wait();
    const int e = find_event(blk_start, E, blockIdx.x);
    const EventHdr& h = hdr[e];
    const int64_t p0 = (int64_t)(blockIdx.x - blk_start[e]) * kBuildPtsPerBlock;
    const int np = (int)min((int64_t)kBuildPtsPerBlock, h.n - p0);
    if (!staged && np > 0) stage_floats(sm, h.refs + p0 * D, np * D, pad);
    __syncthreads();
    const int i = threadIdx.x;
    if (i >= np) return;
    const StagedRow p{sm, i * D, pad};
    int c = 0;
    if (check_finite) {
        bool bad = false;
        for (int k = 0; k < D; ++k) bad |= !isfinite(p[k]);
        if (bad) atomicOr(status, kStatusNonFinite);
    }
    if (h.valid) c = point_cell(p, h);
    const int64_t gi = h.pt_off + p0 + i;
    cid[gi] = c;
    rnk[gi] = atomicAdd(counts + h.cell_off + c, 1);
}

// Slot maps and cell-sorted coordinates: each point's slot (its cell's start
// plus its rank), the slot's original index and cell, and the point's row of
// DP floats (zero padding) written with 16-byte stores (one 32-byte sector
// for D <= 8); the input rows are staged in shared memory with 16-byte loads.
// An odd event's padding slot gets NaN coordinates: never within any radius.
__global__ void __launch_bounds__(kBuildPtsPerBlock) k_scatter(const EventHdr* hdr,
                                                               const int32_t* blk_start, int E,
                                                               int D, int DP,
                                                               const int32_t* cstart,
                                                               const int32_t* cid,
                                                               const int32_t* rnk, float* pts,
                                                               int32_t* perm, int32_t* cell,
                                                               EarlyPts ep) {
    pdl_trigger();
    extern __shared__ float sm[];
    const bool pad = (D & 3) == 0;
    const bool staged = stage_early(sm, ep, D, pad);
    pdl_wait();
    const int e = find_event(blk_start, E, blockIdx.x);
    const EventHdr& h = hdr[e];
    const int64_t p0 = (int64_t)(blockIdx.x - blk_start[e]) * kBuildPtsPerBlock;
    const int np = (int)min((int64_t)kBuildPtsPerBlock, h.n - p0);
    if (p0 == 0 && threadIdx.x == 0 && (h.n & 1)) {
        const int64_t slot = h.pt_off + h.n;
        perm[slot] = -1;
        cell[slot] = 0;
        const float nan = __int_as_float(0x7fc00000);
        float4* dst = reinterpret_cast<float4*>(pts + slot * DP);
        for (int j = 0; j < DP / 4; ++j) dst[j] = make_float4(nan, nan, nan, nan);
    }
    if (!staged && np > 0) stage_floats(sm, h.refs + p0 * D, np * D, pad);
    __syncthreads();
    const int i = threadIdx.x;
    if (i >= np) return;
    const int64_t gi = h.pt_off + p0 + i;
    const int c = cid[gi];
    const int64_t slot = (int64_t)cstart[h.cell_off + c] + rnk[gi];
    perm[slot] = (int32_t)(p0 + i);
    cell[slot] = c;
    const StagedRow src{sm, i * D, pad};
    float4* dst = reinterpret_cast<float4*>(pts + slot * DP);
    for (int j = 0; j < DP / 4; ++j) {
        float4 v;
        v.x = 4 * j + 0 < D ? src[4 * j + 0] : 0.f;
        v.y = 4 * j + 1 < D ? src[4 * j + 1] : 0.f;
        v.z = 4 * j + 2 < D ? src[4 * j + 2] : 0.f;
        v.w = 4 * j + 3 < D ? src[4 * j + 3] : 0.f;
        dst[j] = v;
    }
}

// Per row of cells (all gridded coordinates but the fastest fixed): number of
// query tasks.  A task is the intersection of the row's slot range with a
// window of W slots; windows start at the row's first slot rounded down to a
// multiple of A (A = 1 for the 16-query warp tasks of the grid path, A = 8 for
// the 128-query tensor-core tiles, whose operand rows come in groups of 8).
// Entry i of the cell arrays doubles as row slot i.
__device__ __forceinline__ void row_slots(const EventHdr& h, const int32_t* cstart, int64_t row,
                                          int32_t& base, int32_t& cnt) {
    if (h.valid) {
        const int64_t c0 = h.cell_off + row * h.dims[0];
        base = cstart[c0];
        cnt = cstart[c0 + h.dims[0]] - base;
    } else {
        // invalid event: all its queries in one row (they get empty rows)
        base = (int32_t)h.pt_off;
        cnt = row == 0 ? (int32_t)h.n : 0;
    }
}

__global__ void k_rowtasks(const EventHdr* hdr, const int64_t* cell_off, int E, int64_t i0,
                           int64_t i1, const int32_t* cstart, int32_t* rtask, int W, int A,
                           int path_filter) {
    pdl_trigger();
    pdl_wait();
    const int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= i1) return;
    const int e = find_event64(cell_off, E, i);
    const EventHdr& h = hdr[e];
    const int64_t row = i - cell_off[e];
    int64_t nrows = 1;   // rows: every gridded coordinate but the fastest
    for (int a = 1; a < kMaxAxes && h.valid; ++a) nrows *= h.dims[a];
    int32_t nt = 0;
    // events another launch of a mixed batch queries get no tasks
    if (row < nrows && (path_filter < 0 || h.path == path_filter)) {
        int32_t base, cnt;
        row_slots(h, cstart, row, base, cnt);
        if (cnt > 0) {
            const int32_t w0 = base & ~(A - 1);
            nt = (base + cnt - w0 + W - 1) / W;
        }
    }
    rtask[i] = nt;
}

__global__ void k_emit(const EventHdr* hdr, const int64_t* cell_off, int E, int64_t i0,
                       int64_t i1, const int32_t* cstart, const int32_t* rtask_start,
                       const int32_t* rtask_count_src, Task* tasks, int64_t task_cap, int W,
                       int A, int32_t* status) {
    pdl_trigger();
    pdl_wait();
    const int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= i1) return;
    const int e = find_event64(cell_off, E, i);
    const EventHdr& h = hdr[e];
    const int64_t row = i - cell_off[e];
    const int32_t t0 = rtask_start[i];
    const int32_t t1 = (i + 1 < i1) ? rtask_start[i + 1] : rtask_count_src[0];
    if (t1 <= t0) return;
    int32_t base, cnt;
    row_slots(h, cstart, row, base, cnt);
    const int32_t w0 = base & ~(A - 1);
    for (int32_t t = t0; t < t1; ++t) {
        if (t >= task_cap) {   // never with the tensor-core path's capacity; guarded all the same
            atomicOr(status, kStatusCapacity);
            return;
        }
        const int32_t ws = w0 + (t - t0) * W;
        const int32_t a = max(ws, base);
        const int32_t b = min(ws + W, base + cnt);
        Task tk;
        tk.qslot = a;
        tk.nq = b - a;
        tk.ev = e;
        tk.row = (int32_t)row;
        tasks[t] = tk;
    }
}

void enqueue_tasks(GridBufs& g, int W, int A, Task* out, int64_t out_cap, int32_t* count_out,
                   int32_t* d_status, cudaStream_t st, int path_filter, int64_t i0, int64_t i1) {
    if (i1 < 0) i1 = g.L;
    i0 = std::min(std::max<int64_t>(i0, 0), i1);
    const int64_t n = i1 - i0;
    const unsigned nb = (unsigned)std::max<int64_t>(1, ceil_div(n, 256));
    launch_pdl(k_rowtasks, dim3(nb), dim3(256), 0, st, g.hdr, g.cell_off, g.E, i0, i1, g.cstart,
               g.rtask, W, A, path_filter);
    // the scan of the range's task counts gives each row its first task
    enqueue_scan(g.rtask + i0, n, g.parts, count_out, st);
    launch_pdl(k_emit, dim3(nb), dim3(256), 0, st, g.hdr, g.cell_off, g.E, i0, i1, g.cstart, g.rtask,
               count_out, out, out_cap, W, A, d_status);
}

// ------------------------------------------------------------------ scan
// Exclusive prefix scan of int32 in place (three phases: per-block totals,
// scan of the totals, per-block scan with offset).  Inside a block each thread
// scans kScanItems consecutive values, then warp shuffles scan the thread
// totals and a second warp pass scans the warp totals.

constexpr int kScanThreads = 256;
constexpr int kScanItems = kScanChunk / kScanThreads;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* warp_tot,
                                                        int32_t* block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < (kScanThreads / 32) ? warp_tot[lane] : 0;
        int32_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = z - w;
        if (lane == 31) *block_total = z;
    }
    __syncthreads();
    return x - v + warp_tot[warp];
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* data, int64_t n,
                                                              int32_t* parts) {
    pdl_trigger();
    pdl_wait();
    __shared__ int32_t red[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    int32_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) s += data[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int32_t t = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) parts[blockIdx.x] = t;
    }
}

// Shared-memory slot of chunk entry i: one padding word per 32 entries, so
// that both the coalesced pass (entry k * 256 + t on thread t) and the
// per-thread pass (entries 8t .. 8t + 7 on thread t) touch 32 distinct banks
// per warp access.
__device__ __forceinline__ int scan_slot(int i) { return i + (i >> 5); }
constexpr int kScanSlots = kScanChunk + kScanChunk / 32;

// Scan one chunk of kScanChunk values in place with an added offset.
__device__ void scan_chunk(int32_t* data, int64_t n, int64_t base, int32_t offset,
                           int32_t* total_out) {
    __shared__ int32_t buf[kScanSlots];
    __shared__ int32_t warp_tot[kScanThreads / 32];
    __shared__ int32_t btot;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        buf[scan_slot(k * kScanThreads + threadIdx.x)] = i < n ? data[i] : 0;
    }
    __syncthreads();
    int32_t v[kScanItems];
    int32_t t = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = buf[scan_slot(threadIdx.x * kScanItems + k)];
        t += v[k];
    }
    int32_t ex = block_exclusive_scan(t, warp_tot, &btot) + offset;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        buf[scan_slot(threadIdx.x * kScanItems + k)] = ex;
        ex += v[k];
    }
    __syncthreads();
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) data[i] = buf[scan_slot(k * kScanThreads + threadIdx.x)];
    }
    if (total_out && threadIdx.x == 0) *total_out = btot + offset;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_single(int32_t* data, int64_t n,
                                                              int32_t* total) {
    pdl_trigger();
    pdl_wait();
    scan_chunk(data, n, 0, 0, total);
}

// Down pass.  summed == 0: block b first sums the partials of the blocks
// before it (used while there are at most kScanSumParts of them: at most 16
// L2 reads per thread, cheaper than a launch of the one-block partials scan),
// then scans its chunk with that offset; the last block also writes the
// total.  summed == 1: the partials were already scanned (k_scan_parts).
constexpr int kScanSumParts = 4096;

__global__ void __launch_bounds__(kScanThreads) k_scan_down(int32_t* data, int64_t n,
                                                            const int32_t* parts, int32_t* total,
                                                            int summed) {
    pdl_trigger();
    pdl_wait();
    if (summed) {
        scan_chunk(data, n, (int64_t)blockIdx.x * kScanChunk, parts[blockIdx.x], nullptr);
        return;
    }
    __shared__ int32_t red[kScanThreads / 32];
    __shared__ int32_t offset;
    int32_t v = 0;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += kScanThreads) v += parts[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int32_t t = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) offset = t;
    }
    __syncthreads();
    scan_chunk(data, n, (int64_t)blockIdx.x * kScanChunk, offset,
               blockIdx.x == gridDim.x - 1 ? total : nullptr);
}

// One CTA: exclusive scan of the nb partials in place, chunk after chunk with
// a running carry; writes the grand total.
__global__ void __launch_bounds__(kScanThreads) k_scan_parts(int32_t* parts, int64_t nb,
                                                             int32_t* total) {
    pdl_trigger();
    pdl_wait();
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanChunk) {
        const int32_t c = carry;
        __shared__ int32_t ctot;
        scan_chunk(parts, nb, base, c, &ctot);
        __syncthreads();
        if (threadIdx.x == 0) carry = ctot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

int64_t scan_parts_needed(int64_t n) { return std::max<int64_t>(1, ceil_div(n, kScanChunk)); }

void enqueue_scan(int32_t* data, int64_t n, int32_t* parts, int32_t* total, cudaStream_t st) {
    const int64_t nb = scan_parts_needed(n);
    if (nb == 1) {
        launch_pdl(k_scan_single, dim3(1), dim3(kScanThreads), 0, st, data, n, total);
        return;
    }
    launch_pdl(k_scan_reduce, dim3((unsigned)nb), dim3(kScanThreads), 0, st, data, n, parts);
    if (nb <= kScanSumParts) {
        launch_pdl(k_scan_down, dim3((unsigned)nb), dim3(kScanThreads), 0, st, data, n, parts, total, 0);
    } else {
        launch_pdl(k_scan_parts, dim3(1), dim3(kScanThreads), 0, st, parts, nb, total);
        launch_pdl(k_scan_down, dim3((unsigned)nb), dim3(kScanThreads), 0, st, data, n, parts, total, 1);
    }
}

// ------------------------------------------------------------------ host

// Five gridded axes at a cell edge of about r need about (extent / r)^5
// cells (5.15 M = 17.2 n for the 300k x 8 tracking-like event, whose
// coordinates span [-1.06, 1.06] at r = 0.1), four about (extent / r)^4; the
// budget grows with n so that the cells stay near r on such events (every
// build zeroes and scans the whole budget), and the parameter step falls
// back to one axis fewer when the budget would make five-axis cells too
// coarse.
int64_t cell_cap_for(int64_t n, int naxes) {
    const int64_t per = naxes >= 5 ? 18 : (naxes == 4 ? 2 : 0);
    int64_t c = per ? per * n : n / 2 + 1;
    c = std::max<int64_t>(16384, c);
    return std::min<int64_t>(c, naxes >= 5 ? ((int64_t)1 << 27) : ((int64_t)1 << 24));
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void grid_free(GridBufs& g) {
    tc_free(g);
    rows_free(g);
    if (g.base) cudaFree(g.base);
    if (g.h_pinned) cudaFreeHost(g.h_pinned);
    if (g.h_pinned_free) cudaEventDestroy(g.h_pinned_free);
    g = GridBufs();
}

frnn_status grid_alloc(GridBufs& g, int E, const int64_t* n, int D, std::string& err,
                       const int64_t* caps, int naxes) {
    const int DP = padded_dim(D);
    int64_t n_total = 0, L = 0, nblk = 0, nchunks = 0;
    g.h_hdr.assign(E, EventHdr{});
    g.h_blk_start.assign(E + 1, 0);
    g.h_cell_off.assign(E + 1, 0);
    for (int e = 0; e < E; ++e) {
        const int64_t cap = caps ? caps[e] : cell_cap_for(n[e], naxes);
        EventHdr& h = g.h_hdr[e];
        h.n = n[e];
        h.pt_off = n_total;
        h.cell_off = L;
        h.cell_cap = (int32_t)cap;
        h.qchunk0 = (int32_t)nchunks;
        nchunks += ceil_div(n[e], kChunkQ);
        g.h_blk_start[e] = (int32_t)nblk;
        g.h_cell_off[e] = L;
        n_total += (n[e] + 1) & ~(int64_t)1;   // pair-aligned event regions
        L += cap + 1;
        nblk += std::max<int64_t>(1, ceil_div(n[e], kBuildPtsPerBlock));
    }
    g.h_blk_start[E] = (int32_t)nblk;
    g.h_cell_off[E] = L;
    if (n_total >= INT32_MAX || L >= ((int64_t)1 << 30) ||
        nblk >= INT32_MAX || nchunks >= INT32_MAX) {
        err = "problem too large for one call (points, cells or tasks exceed the limits)";
        return FRNN_ERR_INVALID_ARG;
    }
    g.E = E;
    g.D = D;
    g.DP = DP;
    g.n_total = n_total;
    g.L = L;
    g.nblk = nblk;
    g.nparts = scan_parts_needed(L);
    g.nchunks = nchunks;
    // the buffers are reused only if every region is large enough, the
    // point rows included (a set of a higher dimension needs wider rows)
    const bool fits = g.base && g.cap_n >= n_total && g.cap_DP >= DP && g.cap_L >= L && g.cap_E >= E &&
                      g.cap_blk >= nblk;
    const int64_t cn = std::max<int64_t>(n_total, 1);
    if (!fits) {
        if (g.base) {
            cudaFree(g.base);
            g.base = nullptr;
        }
        size_t off = 0;
        auto take = [&](size_t bytes) {
            size_t o = off;
            off = align_up(off + bytes, 256);
            return o;
        };
        const size_t o_hdr = take(sizeof(EventHdr) * E);
        const size_t o_blk = take(sizeof(int32_t) * (E + 1));
        const size_t o_coff = take(sizeof(int64_t) * (E + 1));
        const size_t o_bbox = take(sizeof(int32_t) * kBBoxStride * kBBoxCopies * E);
        const size_t o_pts = take(sizeof(float) * DP * (cn + kTcRowPad));
        const size_t o_perm = take(sizeof(int32_t) * cn);
        const size_t o_cell = take(sizeof(int32_t) * cn);
        const size_t o_cid = take(sizeof(int32_t) * cn);
        const size_t o_rnk = take(sizeof(int32_t) * cn);
        const size_t o_cst = take(sizeof(int32_t) * L);
        const size_t o_ovf = take(sizeof(Overflow) * cn);
        const size_t o_sc = take(sizeof(int32_t) * kScalars);
        const size_t o_parts = take(sizeof(int32_t) * g.nparts);
        void* base = nullptr;
        cudaError_t ce = cudaMalloc(&base, off);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            err = std::string("cudaMalloc of grid buffers failed: ") + cudaGetErrorString(ce);
            g.cap_n = g.cap_L = g.cap_E = g.cap_blk = 0;
            g.cap_DP = 0;
            return FRNN_ERR_OUT_OF_MEMORY;
        }
        char* b = static_cast<char*>(base);
        g.base = base;
        g.bytes = off;
        g.hdr = reinterpret_cast<EventHdr*>(b + o_hdr);
        g.blk_start = reinterpret_cast<int32_t*>(b + o_blk);
        g.cell_off = reinterpret_cast<int64_t*>(b + o_coff);
        g.bbox = reinterpret_cast<int32_t*>(b + o_bbox);
        g.pts = reinterpret_cast<float*>(b + o_pts);
        g.perm = reinterpret_cast<int32_t*>(b + o_perm);
        g.cell = reinterpret_cast<int32_t*>(b + o_cell);
        g.cid = reinterpret_cast<int32_t*>(b + o_cid);
        g.rnk = reinterpret_cast<int32_t*>(b + o_rnk);
        g.cstart = reinterpret_cast<int32_t*>(b + o_cst);
        g.rtask = nullptr;   // the tensor-core operands carry the task builder's scratch
        g.ovf = reinterpret_cast<Overflow*>(b + o_ovf);
        g.scalars = reinterpret_cast<int32_t*>(b + o_sc);
        g.parts = reinterpret_cast<int32_t*>(b + o_parts);
        g.cap_n = n_total;
        g.cap_DP = DP;
        g.cap_L = L;
        g.cap_E = E;
        g.cap_blk = nblk;
    }
    // page-locked mirror for the per-event tables
    // (laid out like the device tables: header, block starts and cell offsets
    // at the same relative offsets, so one copy uploads all three)
    const size_t hbytes = (size_t)(reinterpret_cast<char*>(g.cell_off) -
                                   reinterpret_cast<char*>(g.hdr)) +
                          sizeof(int64_t) * (E + 1) + 64;
    if (g.h_pinned_bytes < hbytes) {
        if (g.h_pinned) {
            if (g.h_pinned_free) cudaEventSynchronize(g.h_pinned_free);
            cudaFreeHost(g.h_pinned);
            g.h_pinned = nullptr;
        }
        if (cudaMallocHost(&g.h_pinned, hbytes) != cudaSuccess) {
            cudaGetLastError();
            g.h_pinned_bytes = 0;
            err = "cudaMallocHost of grid tables failed";
            return FRNN_ERR_OUT_OF_MEMORY;
        }
        g.h_pinned_bytes = hbytes;
    }
    if (!g.h_pinned_free) cudaEventCreateWithFlags(&g.h_pinned_free, cudaEventDisableTiming);
    return FRNN_OK;
}

// k_init's blocks: four per SM of the GB300's 152, all resident at once, so
// that every block triggers the next kernel at once and the bounding-box
// blocks can stage their points while k_init finishes (2, 4 and 8 per SM
// measured the same build time at 300k x 8, 0.051 ms; the gain over 0.057
// is the early staging)
constexpr unsigned kInitBlocks = 608;

static inline unsigned blocks_for(int64_t n, int t) {
    return (unsigned)std::max<int64_t>(1, ceil_div(n, t));
}

// Cell ids, the cell-start scan, slot maps, coordinates.
static void enqueue_sort(GridBufs& g, size_t smem_pts, int check_finite, int32_t* d_status,
                         cudaStream_t st, EarlyPts ep) {
    const int E = g.E, D = g.D;
    launch_pdl(k_cellid, dim3((unsigned)g.nblk), dim3(kBuildPtsPerBlock), smem_pts, st,
               g.hdr, g.blk_start, E, D, g.cstart, g.cid, g.rnk, check_finite, d_status, ep);
    enqueue_scan(g.cstart, g.L, g.parts, g.scalars + kScCellTotal, st);
    launch_pdl(k_scatter, dim3((unsigned)g.nblk), dim3(kBuildPtsPerBlock), smem_pts, st,
               g.hdr, g.blk_start, E, D, g.DP, g.cstart, g.cid, g.rnk, g.pts, g.perm, g.cell, ep);
    // no task list: the grid query takes chunks of kChunkQ slots in slot order
}

frnn_status enqueue_build(GridBufs& g, const float* const* refs, const BuildOpts& o,
                          const GridBufs* params_from, int32_t* d_status, cudaStream_t st,
                          bool capturing, std::string& err) {
    const int E = g.E, D = g.D;
    for (int e = 0; e < E; ++e) {
        g.h_hdr[e].refs = refs[e];
        g.h_hdr[e].valid = 1;
    }
    // one event outside a capture: k_init writes the tables from its
    // arguments (no copy on the stream, so the chain stays one run of
    // programmatically dependent kernels)
    OneEventTables t1{};
    if (E == 1 && !capturing) {
        t1.hdr = g.h_hdr[0];
        t1.cell_end = g.h_cell_off[1];
        t1.nblk = g.h_blk_start[1];
        t1.set = 1;
    } else {
    // upload the per-event tables through the pinned mirror (wait until the
    // previous upload from it has been consumed)
    if (!capturing) cudaEventSynchronize(g.h_pinned_free);
    // the three tables are adjacent on the device: mirror that layout in the
    // pinned buffer and upload them with one copy
    char* hp = static_cast<char*>(g.h_pinned);
    const size_t s_hdr = sizeof(EventHdr) * E;
    const size_t s_blk = sizeof(int32_t) * (E + 1);
    const size_t s_coff = sizeof(int64_t) * (E + 1);
    const size_t o_blk = reinterpret_cast<char*>(g.blk_start) - reinterpret_cast<char*>(g.hdr);
    const size_t o_coff = reinterpret_cast<char*>(g.cell_off) - reinterpret_cast<char*>(g.hdr);
    memcpy(hp, g.h_hdr.data(), s_hdr);
    memcpy(hp + o_blk, g.h_blk_start.data(), s_blk);
    memcpy(hp + o_coff, g.h_cell_off.data(), s_coff);
    cudaMemcpyAsync(g.hdr, hp, o_coff + s_coff, cudaMemcpyHostToDevice, st);
    if (!capturing) cudaEventRecord(g.h_pinned_free, st);
    }

    const int32_t bbmin = host_float_to_ordered(INFINITY);
    const int32_t bbmax = host_float_to_ordered(-INFINITY);
    const int64_t init_n = std::max<int64_t>(g.L, (int64_t)E * kBBoxCopies * kBBoxStride);
    launch_pdl(k_init, dim3(std::min<unsigned>(blocks_for(init_n, 256), kInitBlocks)), dim3(256), 0, st,
        g.cstart, g.L, g.bbox, E, g.scalars, bbmin, bbmax, t1, g.hdr, g.blk_start, g.cell_off);
    const size_t smem_pts = sizeof(float) * staged_floats(D);
    const EarlyPts ep{t1.hdr.refs, t1.hdr.n, t1.set};
    if (params_from) {
        launch_pdl(k_copy_params, dim3(blocks_for(E, 128)), dim3(128), 0, st, g.hdr, params_from->hdr, E,
                   g.cstart);
    } else {
        launch_pdl(k_bbox, dim3((unsigned)g.nblk), dim3(kBuildPtsPerBlock), smem_pts, st, g.hdr, g.blk_start, E, D,
                   g.bbox, d_status, o.r, o.m, o.axes_mode, o.naxes, g.cstart, ep);
    }
    enqueue_sort(g, smem_pts, params_from ? 1 : 0, d_status, st, ep);
    g.tc_ready = false;     // tensor-core operands describe the previous contents
    g.rows_ready = false;   // so do the row-task kernel's pair copy and tasks
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("grid build launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    return FRNN_OK;
}

// The same build as enqueue_build, for a point set whose per-event tables
// (headers, block starts, cell offsets) some earlier work on the stream has
// already written on the device: nothing is copied from the host.
frnn_status enqueue_build_resident(GridBufs& g, const BuildOpts& o, int32_t* d_status,
                                   cudaStream_t st, std::string& err) {
    const int E = g.E, D = g.D;
    const int32_t bbmin = host_float_to_ordered(INFINITY);
    const int32_t bbmax = host_float_to_ordered(-INFINITY);
    const int64_t init_n = std::max<int64_t>(g.L, (int64_t)E * kBBoxCopies * kBBoxStride);
    launch_pdl(k_init, dim3(std::min<unsigned>(blocks_for(init_n, 256), kInitBlocks)), dim3(256), 0, st,
        g.cstart, g.L, g.bbox, E, g.scalars, bbmin, bbmax, OneEventTables{}, g.hdr, g.blk_start,
        g.cell_off);
    const size_t smem_pts = sizeof(float) * staged_floats(D);
    launch_pdl(k_bbox, dim3((unsigned)g.nblk), dim3(kBuildPtsPerBlock), smem_pts, st, g.hdr, g.blk_start, E, D,
               g.bbox, d_status, o.r, o.m, o.axes_mode, o.naxes, g.cstart, EarlyPts{});
    enqueue_sort(g, smem_pts, 0, d_status, st, EarlyPts{});
    g.tc_ready = false;
    g.rows_ready = false;
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("grid build launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    return FRNN_OK;
}

}  // namespace frnn
