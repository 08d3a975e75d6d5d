// frnn_internal.cuh — device data layout, launch helpers and PTX wrappers
// shared by the library's translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/frnn.h"

namespace frnn {

constexpr int kMaxD = 16;
constexpr int kMaxK = 1024;
constexpr int kMaxAxes = 5;
constexpr int kMaxDimsPerAxis = 1024;   // the grid roundoff proof assumes <= 2^10 cells per axis
constexpr int kTaskQueries = 16;        // task-list granularity of the build's task builder
constexpr int kChunkQ = 16;             // query slots per chunk of the grid query kernel
// neighbour rows of a row of cells, (2m+1)^(naxes-1), that the query kernels
// enumerate (32 per round of a warp): 81 for five axes with m = 1, 125 for
// four with m = 2, 49 for three with m = 3
constexpr int kMaxNbrRows = 128;

// Device status word bits (frnn_sync maps them to frnn_status).
constexpr int kStatusNonFinite = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusCapacity = 4;
// compact (CSR) output: staging rows of kCsrStageW entries per query; a count
// with kCsrSpill set belongs to a row the selection kernel writes itself
constexpr int kCsrStageW = 32;
constexpr int32_t kCsrSpill = 0x40000000;
constexpr int32_t kCsrCountMask = 0x3fffffff;

// Bounded waits: an mbarrier wait gives up after about two seconds of wall
// time (%globaltimer), far above any legitimate wait, with an iteration cap as
// a backstop.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint32_t kSpinLimit = 1u << 30;

// Padded point row: D floats rounded up to a multiple of 4 (16 bytes).
__host__ __device__ constexpr int padded_dim(int D) { return (D + 3) & ~3; }

// Cell-sorted points are stored as rows of DP floats (coordinate k of slot s
// at s * DP + k; the padding coordinates are zero), so the points of any
// slot range form one contiguous, 16-byte aligned block: one bulk copy moves
// a whole range of candidates into shared memory.  Every event's slot range
// starts on an even slot (odd events get one padding slot with NaN
// coordinates), the layout the build's scans and the tensor-core operands use.
__host__ __device__ constexpr int64_t pt_index(int64_t slot, int k, int DP) {
    return slot * DP + k;
}

// Per-event grid header (device-resident, one per event of a build).
struct EventHdr {
    const float* refs;     // caller's [n, D] input (build only)
    int64_t n;             // points in this event
    int64_t pt_off;        // first sorted slot of this event (global slot numbering)
    int64_t cell_off;      // first entry of this event in the cell arrays (cap + 1 entries)
    int32_t cell_cap;      // cells allowed for this event
    int32_t ncells;        // product of dims (written by the parameter step)
    int32_t naxes;         // gridded axes (1..5); preset by the host: requested count (0: default)
    int32_t m;             // cell multiple: neighbours are within +-m cells per gridded axis
    int32_t valid;         // 0 if a coordinate was non-finite
    int32_t axes[kMaxAxes];   // gridded coordinate indices; axes[0] varies fastest
    int32_t dims[kMaxAxes];   // cells per gridded axis (1 for unused axes)
    float lo[kMaxAxes];       // per-axis minimum coordinate
    float hi[kMaxAxes];       // per-axis maximum coordinate
    float inv_h;           // 1 / cell edge (float; the value the cell ids use)
    int32_t path;          // batched queries: 0 = grid scan, 1 = tensor-core pre-filter
    int32_t qchunk0;       // first query chunk (kChunkQ slots) of this event in its point set
    float ctr[16];         // per-dimension centre of the bounding box (tensor-core operands)
    // query outputs for batched self-queries (row = original point index)
    int32_t* counts;
    int32_t* idx;
    float* dist2;
};

// One warp task: up to 16 consecutive cell-sorted query slots lying in one
// row of cells (all gridded coordinates but the fastest equal).
struct Task {
    int32_t qslot;   // first query slot (global)
    int32_t nq;      // queries in the task (1..16 for warp tasks, 1..128 for tensor-core tiles)
    int32_t ev;      // event index
    int32_t row;     // row index within the event: c1 + dims[1] * (c2 + dims[2] * (c3 + ...))
};

// Neighbour rows of a row of cells.  A row fixes every gridded coordinate but
// the fastest (c0); its neighbours are the rows whose coordinates c1..c4 each
// differ by at most m.  Neighbour l (0 <= l < neighbour_rows(h)) takes the
// offsets given by the base-(2m+1) digits of l, minus m.  Returns false if
// that row lies outside the grid, else its first cell index.
__host__ __device__ inline int neighbour_rows(const EventHdr& h) {
    const int side = 2 * h.m + 1;
    int n = 1;
    for (int a = 1; a < h.naxes; ++a) n *= side;
    return n;
}
__device__ __forceinline__ bool neighbour_row(const EventHdr& h, int row, int l,
                                              int64_t& first_cell) {
    const int side = 2 * h.m + 1;
    int64_t lin = 0, stride = 1;
    bool ok = true;
#pragma unroll
    for (int a = 1; a < kMaxAxes; ++a) {
        const int da = h.dims[a];
        const int c = row % da;
        row /= da;
        int d = 0;
        if (a < h.naxes) {
            d = (l % side) - h.m;
            l /= side;
        }
        const int cc = c + d;
        ok = ok && cc >= 0 && cc < da;
        lin += (int64_t)cc * stride;
        stride *= da;
    }
    first_cell = h.cell_off + lin * h.dims[0];
    return ok;
}

// Overflowed query (degree > K): handled by the exact selection kernel.
struct Overflow {
    int32_t qslot;
    int32_t ev;
};

// Everything the query kernels need, passed by value.
struct QueryArgs {
    const EventHdr* ev;          // per-event headers (reference grids)
    const EventHdr* qev;         // per-event headers of the query set (== ev for self-queries)
    int32_t nev;                 // events
    int32_t nchunks;             // query chunks over all events
    const Task* tasks;           // row-task kernel: 16-query warp tasks of the query set
    const int32_t* ntasks;       // row-task kernel: device scalar, number of tasks
    const float* qpts;           // cell-sorted query coordinates [*, DP]
    const int32_t* qperm;        // query slot -> original query index (within its event)
    const int32_t* qcell;        // query slot -> local cell id
    const float* rpts;           // cell-sorted reference coordinates [*, DP]
    const int32_t* rperm;        // reference slot -> original index (within its event)
    const int32_t* cstart;       // reference cell starts (global slots), per event cap+1
    int32_t* counts;             // single-event outputs (NULL: use the per-event ones)
    int32_t* idx;
    float* dist2;
    float r2;                    // fl(r * r)
    float r2_screen;             // row-task kernel: r2 (1 + 2^-16) rounded up, the packed screen's bound
    int32_t K;
    int32_t self;                // 1: query slot == reference slot is excluded
    int32_t D;
    int32_t* task_counter;       // device scalar: chunk counter, zero at launch
    int32_t* status;             // device status word
    Overflow* ovf;               // overflow list
    int32_t* ovf_count;          // device scalar
    int32_t ovf_cap;
    int32_t* ovf_done;           // device scalar: finished blocks of the selection kernel
    int32_t reset_ovf;           // selection kernel: 1 = clear the overflow list when done
    int32_t exit_dims;           // dims summed before the warp early-exit vote
    int32_t path_filter;         // -1: every event; else only events whose path matches
    // compact output.  csr = 1: rows go to idx/dist2 at row * kCsrStageW (no
    // padding) and counts get kCsrSpill for rows left to the selection kernel.
    // Selection kernel mode: 0 dense rows, 1 count only (counts | kCsrSpill and
    // degree), 2 rows at row_off[query].
    int32_t csr;
    int32_t ovf_mode;
    int32_t* degree;             // optional full degree per query (csr)
    const int64_t* row_off;      // CSR row offsets (ovf_mode 2)
    int64_t row_cap;             // entries idx / dist2 hold (ovf_mode 2): rows past it are skipped
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completion signalled on an mbarrier.
// dst, src 16-byte aligned; bytes a positive multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// try_wait suspends the thread until the phase completes or a time hint
// (here 20 us) elapses, so waiting warps do not spin on the issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: returns false (and the caller records a timeout) if the phase
// did not complete within limit_ns of %globaltimer time (or kSpinLimit polls).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1; it < kSpinLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 7u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization (launch_pdl) may be scheduled while its predecessor on the
// stream is still running: pdl_trigger() lets the successor launch,
// pdl_wait() blocks until the predecessor grid has completed and its memory
// writes are visible.  Every kernel of the build and query chain calls both
// before touching its inputs; for a kernel launched the ordinary way they do
// nothing.  This hides the launch gap between the chain's short kernels.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Ordered-int encoding of float for atomic min/max (monotone in float order).
__device__ __forceinline__ int32_t float_to_ordered(float f) {
    int32_t i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_to_float(int32_t i) {
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}
inline int32_t host_float_to_ordered(float f) {
    int32_t i;
    memcpy(&i, &f, 4);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__host__ __device__ constexpr int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------ per-thread sort
// A thread's neighbour list lives in shared memory as a column of a
// transposed table: entry e at d2[e * stride], idx[e * stride].  With perm,
// idx holds the reference's sorted slot and sorting maps it to the original
// index (the tie-break key); without, idx already holds the original index.
// The sort builds 64-bit keys (d2 bits << 32 | index) (d2 >= +0, so the
// unsigned order of the keys is the (d2, index) order) and runs a fixed
// bitonic network in registers: no data-dependent branches, so the lanes of
// a warp stay converged.
template <int S>
__device__ __forceinline__ void sort_list_net(float* d2, int32_t* idx, int stride, int cnt,
                                              const int32_t* perm) {
    uint64_t k[S];
#pragma unroll
    for (int e = 0; e < S; ++e) {
        k[e] = ~0ull;
        if (e < cnt) {
            const int32_t slot = idx[e * stride];
            k[e] = ((uint64_t)__float_as_uint(d2[e * stride]) << 32) |
                   (uint32_t)(perm ? perm[slot] : slot);
        }
    }
#pragma unroll
    for (int kk = 2; kk <= S; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & kk) == 0;
                    const uint64_t x = k[i], y = k[l];
                    const bool sw = up ? (x > y) : (x < y);
                    k[i] = sw ? y : x;
                    k[l] = sw ? x : y;
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < S; ++e) {
        if (e < cnt) {
            d2[e * stride] = __uint_as_float((uint32_t)(k[e] >> 32));
            idx[e * stride] = (int32_t)(uint32_t)k[e];
        }
    }
}

// Sort one thread's list of cnt <= 32 entries (warp-uniform network size).
__device__ __forceinline__ void sort_list(float* d2, int32_t* idx, int stride, int cnt,
                                          const int32_t* perm) {
    const unsigned full = __activemask();
    int mx = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(full, mx, o));
    if (mx <= 1) {
        if (cnt == 1 && perm) idx[0] = perm[idx[0]];
    } else if (mx <= 4) {
        sort_list_net<4>(d2, idx, stride, cnt, perm);
    } else if (mx <= 8) {
        sort_list_net<8>(d2, idx, stride, cnt, perm);
    } else if (mx <= 16) {
        sort_list_net<16>(d2, idx, stride, cnt, perm);
    } else {
        sort_list_net<32>(d2, idx, stride, cnt, perm);
    }
}

}  // namespace frnn
