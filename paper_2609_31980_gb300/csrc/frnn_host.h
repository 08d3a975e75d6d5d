// frnn_host.h — host-side structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "frnn_internal.cuh"

namespace frnn {

// Device buffers of one (possibly multi-event) cell-sorted point set: the
// reference grid of frnn_build_grid / frnn_query_batched, or the binned query
// set of a cross-set frnn_query.  One cudaMalloc block, carved into arrays.
struct GridBufs {
    int E = 0;              // events
    int D = 0, DP = 0;      // dimensions, padded row length (floats)
    int64_t n_total = 0;    // points over all events
    int64_t L = 0;          // cell-array entries: sum over events of (cell_cap + 1)
    int64_t nblk = 0;       // blocks of the per-point build kernels
    int64_t nparts = 0;     // scan partial sums needed
    int64_t nchunks = 0;    // query chunks (kChunkQ slots) over all events
    // the last query left its overflow list for a compact fill pass that has
    // not run: the next query clears the list first
    mutable bool ovf_stale = false;

    // allocation (reused when large enough)
    void* base = nullptr;
    size_t bytes = 0;
    int64_t cap_n = 0, cap_L = 0, cap_E = 0, cap_blk = 0;
    int cap_DP = 0;         // row width the point rows were carved for
    void* h_pinned = nullptr;      // page-locked host mirror of the small tables
    size_t h_pinned_bytes = 0;
    cudaEvent_t h_pinned_free = nullptr;   // last upload from the mirror has run

    // device arrays
    EventHdr* hdr = nullptr;       // [E]
    int32_t* blk_start = nullptr;  // [E + 1] first build block of each event
    int64_t* cell_off = nullptr;   // [E + 1] first cell-array entry of each event
    int32_t* bbox = nullptr;       // [E * kBBoxCopies * kBBoxStride] ordered-int min / max / flag
    float* pts = nullptr;          // [n_total * DP] cell-sorted coordinates
    int32_t* perm = nullptr;       // [n_total] slot -> original index in its event
    int32_t* cell = nullptr;       // [n_total] slot -> local cell id
    int32_t* cid = nullptr;        // [n_total] input order -> local cell id
    int32_t* rnk = nullptr;        // [n_total] input order -> rank inside its cell
    int32_t* cstart = nullptr;     // [L] cell counts, then (scanned) global start slots
    int32_t* rtask = nullptr;      // [L] per-row task counts, then task starts (tensor-core tiles)
    Overflow* ovf = nullptr;       // [n_total]
    int32_t* scalars = nullptr;    // [kScalars] counters (below)
    int32_t* parts = nullptr;      // [nparts] scan partial sums

    // tensor-core operands (allocated on the first tensor-core query)
    bool tc_ready = false;
    void* tc_base = nullptr;
    size_t tc_bytes = 0;
    int64_t tc_cap_rows = 0, tc_cap_tasks = 0, tc_cap_E = 0, tc_cap_L = 0;
    int32_t* tc_rtask = nullptr;   // [L] the task builder's per-row scratch
    int tc_K = 0;                  // operand row length (bf16 elements, multiple of 16)
    uint16_t* tcA = nullptr;       // [rows] query-role rows, core-matrix layout
    uint16_t* tcB = nullptr;       // [rows] candidate-role rows, core-matrix layout
    float* tcn = nullptr;          // [rows] squared norm of the centred split coordinates
    int32_t* tcnu = nullptr;       // [E] ordered-int max norm per event
    Task* tc_tasks = nullptr;      // 128-query tasks

    // row-task kernel (grids of up to four axes): pair-interleaved copy of
    // the points and 16-query tasks, made at query time after each build
    bool rows_ready = false;
    void* rows_base = nullptr;
    size_t rows_bytes = 0;
    int64_t rows_cap_n = 0, rows_cap_tasks = 0, rows_cap_L = 0;
    int rows_cap_DP = 0;            // row width the pair copy was sized for
    float* ppts = nullptr;          // [n_total * DP] pair-interleaved coordinates
    Task* row_tasks = nullptr;      // [rows_cap_tasks]
    int32_t* rows_rtask = nullptr;  // [L] the task builder's per-row scratch

    // host copies
    std::vector<EventHdr> h_hdr;
    std::vector<int32_t> h_blk_start;
    std::vector<int64_t> h_cell_off;
};

constexpr int kBBoxStride = 34;      // 16 minima, 16 maxima, non-finite flag, finished blocks
constexpr int kBBoxCopies = 32;      // copies of each event's box (spread the atomics)
constexpr int kScanChunk = 2048;     // entries per block of the exclusive scan
constexpr int kBuildPtsPerBlock = 256;
// indices into GridBufs::scalars
constexpr int kScNTasks = 0;        // number of warp tasks
constexpr int kScCellTotal = 1;     // total of the cell-count scan (= n_total)
constexpr int kScTaskCounter = 2;   // chunk counter of the grid query kernel
constexpr int kScOvfCount = 3;      // overflowed queries
constexpr int kScTcCounter = 4;     // task counter of the tensor-core kernel
constexpr int kScTcTasks = 5;      // number of tensor-core tasks
constexpr int kScOvfDone = 6;       // finished blocks of the selection kernel
constexpr int kScalars = 16;
constexpr int kTcRowPad = 512;      // rows readable past the last slot (chunk round-up)

// Cells allowed for an n-point event gridded over naxes coordinates (the
// parameter step enlarges the cells when the grid would need more).
int64_t cell_cap_for(int64_t n, int naxes);

// Compute the layout for E events of sizes n[e] and allocate (or reuse).
// caps (optional): per-event cell capacities (a query set binned with a
// reference grid's parameters must use that grid's capacities); otherwise
// cell_cap_for(n[e], naxes).
frnn_status grid_alloc(GridBufs& g, int E, const int64_t* n, int D, std::string& err,
                       const int64_t* caps = nullptr, int naxes = kMaxAxes);
void grid_free(GridBufs& g);

struct BuildOpts {
    float r = 0.f;          // grid radius
    int m = 1;              // cell multiple
    int axes_mode = 0;      // 0: last axes, 1: widest axes
    int naxes = 0;          // gridded axes requested (at most D, kMaxAxes); 0 = automatic
};

// Enqueue a full build (bounding boxes, parameters, binning, counting sort,
// tasks).  refs[e] = event e's [n_e, D] device input.  If params_from is not
// NULL the grid parameters are copied from it (cross-set query binning) instead
// of being derived from this set's bounding box.  capturing: the stream is
// being captured into a CUDA graph (no host-side event waits or records).
frnn_status enqueue_build(GridBufs& g, const float* const* refs, const BuildOpts& o,
                          const GridBufs* params_from, int32_t* d_status, cudaStream_t st,
                          bool capturing, std::string& err);

// Task list: windows of W slots aligned to A within each row of cells
// (at most out_cap tasks; beyond it the status word records a capacity error).
// path_filter >= 0: only rows of events whose path is path_filter get tasks
// (a mixed batch queries its other events in other launches).  [i0, i1):
// the cell-array entries (rows) considered (i1 < 0: to the end); a batch
// ordered by path passes the range of its events of this path.
void enqueue_tasks(GridBufs& g, int W, int A, Task* out, int64_t out_cap, int32_t* count_out,
                   int32_t* d_status, cudaStream_t st, int path_filter = -1, int64_t i0 = 0,
                   int64_t i1 = -1);

// The build for per-event tables already resident on the device.
frnn_status enqueue_build_resident(GridBufs& g, const BuildOpts& o, int32_t* d_status,
                                   cudaStream_t st, std::string& err);

// Exclusive scan of n int32 values in place; the total goes to *total.
void enqueue_scan(int32_t* data, int64_t n, int32_t* parts, int32_t* total, cudaStream_t st);
int64_t scan_parts_needed(int64_t n);

// Query launch (grid path).
struct QueryLaunch {
    const GridBufs* qset;   // query slots and tasks
    const GridBufs* rset;   // reference grid
    float r2;
    int K;
    int self;
    int exit_dims;          // 0 = default
    int stage = 0;          // grid query candidate staging: 0 lanes load rows, 1 bulk copies
    int kernel = 0;         // grid scan: 0 chunks (query.cu), 1 row tasks (query_rows.cu)
    int32_t* counts;        // single event outputs, or NULL to use the event headers'
    int32_t* idx;
    float* dist2;
    int32_t* d_status;
    int num_sms;
    unsigned long long* tc_stats = nullptr;   // [2]: pre-filter survivors, exact accepts
    int path_filter = -1;                     // batched: only events of this path
    int64_t chunk_end = -1;                   // chunk scan: chunks [0, chunk_end) (-1: all)
    cudaEvent_t kev[2] = {nullptr, nullptr};  // optional: recorded around the main kernel
    // compact output (csr.cu): staging mode of the main kernels and the
    // selection kernel's mode (0 dense, 1 count, 2 rows at row_off)
    int csr = 0;
    int ovf_mode = 0;
    int32_t* degree = nullptr;
    const int64_t* row_off = nullptr;
    int64_t row_cap = INT64_MAX;   // compact rows: entries the output holds
};
frnn_status enqueue_grid_query(const QueryLaunch& q, cudaStream_t st, std::string& err);
// Row-task kernel: allocate (outside any capture) and build (enqueued) the
// pair-interleaved copy and 16-query tasks of a point set; the launch itself
// (called by enqueue_grid_query when q.kernel == 1, inputs prepared).
frnn_status rows_reserve(GridBufs& g, std::string& err);
// [i0, i1): cell-array range of the events to prepare, [s0, s1): their slots
// (negative ends: to the end of the set)
frnn_status rows_prepare(GridBufs& g, int32_t* d_status, cudaStream_t st, std::string& err,
                         int path_filter = -1, int64_t i0 = 0, int64_t i1 = -1, int64_t s0 = 0,
                         int64_t s1 = -1);
void rows_free(GridBufs& g);
frnn_status enqueue_row_query(const QueryLaunch& q, const QueryArgs& a, cudaStream_t st,
                              std::string& err);
// The selection kernel alone over the rows the last query of q.qset listed
// (compact output, second pass: q.ovf_mode 2, q.row_off).
frnn_status enqueue_overflow_only(const QueryLaunch& q, cudaStream_t st, std::string& err);
// Compact output (csr.cu): offsets[0..M] from the marked counts; the gather
// of the staged rows.  parts: csr_parts_needed(M) int64 scratch.
int64_t csr_parts_needed(int64_t M);
void enqueue_csr_offsets(const int32_t* cnt, int64_t M, int64_t* parts, int64_t* offsets,
                         cudaStream_t st);
// cap: entries idx / dist2 hold; entries at or past it are not written.
// [row0, row1): the rows gathered (row0 a multiple of 32; row1 < 0: to M).
void enqueue_csr_gather(const int32_t* cnt, const int64_t* offsets, const int32_t* sidx,
                        const float* sd2, int64_t M, int32_t* idx, float* dist2, int num_sms,
                        cudaStream_t st, int64_t cap = INT64_MAX, int64_t row0 = 0,
                        int64_t row1 = -1);

// Tensor-core path: prepare operands (and 128-query tasks) of a point set.
// center_src: the grid whose per-event centres the operands use (the
// reference grid; the set itself for self-queries).
frnn_status tc_prepare(GridBufs& g, const GridBufs& center_src, int32_t* d_status, cudaStream_t st,
                       std::string& err, int path_filter = -1, int64_t i0 = 0, int64_t i1 = -1);
frnn_status enqueue_tc_query(const QueryLaunch& q, cudaStream_t st, std::string& err);
frnn_status tc_reserve(GridBufs& g, std::string& err);
void tc_free(GridBufs& g);
frnn_status enqueue_overflow(const QueryArgs& a, int num_sms, cudaStream_t st, std::string& err);

// Context helpers for the serving loop (defined with the context, api.cu).
void ctx_copy_tuning(frnn_ctx* dst, const frnn_ctx* src);
// Launch a kernel with programmatic stream serialization (see pdl_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Device address of a page-locked host buffer, or NULL (pageable / unknown).
void* mapped_host(const void* p);
// diag.cu: one warp waits (bounded by limit_ns) on a barrier nothing completes
cudaError_t launch_wait_timeout(uint64_t limit_ns, int32_t* status, cudaStream_t st);
// Grow the context's batched workspace (and the tensor-core operands when the
// path would be taken) to hold E events of n points each, so later batched
// calls of at most E events of at most n points allocate nothing.
frnn_status ctx_reserve_batch(frnn_ctx* ctx, int E, int64_t n, int D, int K, unsigned flags);
void ctx_set_error(frnn_ctx* ctx, const char* msg);

}  // namespace frnn
