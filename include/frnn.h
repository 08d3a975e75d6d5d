/*
 * frnn.h — C ABI of the GB300 (sm_103a) exact fixed-radius nearest-neighbour
 * library.
 *
 * The operation is the paper's Eq. 1 (Sec. 1): for query points x_i and
 * reference points x_j in R^D,
 *
 *     N_r(i) = { j : ||x_i - x_j||_2 <= r },
 *
 * keeping at most K neighbours in distance order.  Membership and distances
 * follow one fixed float32 contract, identical to a brute-force scan:
 *
 *     s = +0;  for k = 0..D-1:  d = fl(q_k - p_k);  s = fl(s + fl(d*d));
 *     j in N_r(i)  <=>  s <= fl(r*r)
 *
 * (round to nearest, dimensions in index order, no fused multiply-add; the
 * paper's Sec. 4.2 reports that reordered accumulation changed membership near
 * the radius and was rejected as inexact).  Each result row holds
 * min(degree, K) neighbours sorted by (s, original index) ascending; the rest
 * of the row is padded with index -1 and distance +inf.  Returned distances
 * are the squared distances s, bit for bit.
 *
 * Conventions for every call:
 *   - Pointers marked "device" are CUDA device (or managed) pointers; the
 *     caller owns them and keeps them alive until the work is complete.
 *   - Work is enqueued asynchronously on the context's stream.  Host-side
 *     argument errors are returned at once; device-side errors (non-finite
 *     coordinates, an exceeded internal capacity, a bounded wait that ran out)
 *     are recorded in a device status word and returned by frnn_sync().
 *   - The library owns its contexts, workspaces and grids.
 *   - A context is not thread-safe: use one per host thread.
 *   - Limits: 1 <= D <= 16, 1 <= K <= 1024, 0 <= N, M < 2^31 - 1 (per call,
 *     summed over events for batched calls); r finite with
 *     2^-60 <= r <= 2^60.
 */
#ifndef FRNN_H
#define FRNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum frnn_status {
    FRNN_OK = 0,
    FRNN_ERR_INVALID_ARG = -1,   /* bad pointer, size, D, K, r or flag */
    FRNN_ERR_UNSUPPORTED = -2,   /* valid request this build does not serve */
    FRNN_ERR_OUT_OF_MEMORY = -3, /* a device allocation failed */
    FRNN_ERR_BUDGET = -4,        /* the request does not fit the memory budget */
    FRNN_ERR_NONFINITE = -5,     /* an input coordinate is NaN or +-inf */
    FRNN_ERR_CUDA = -6,          /* a CUDA runtime call failed */
    FRNN_ERR_TIMEOUT = -7,       /* a bounded device-side wait ran out */
    FRNN_ERR_CAPACITY = -8       /* an internal device-side capacity overflowed */
} frnn_status;

/* frnn_query / frnn_query_batched flags */
#define FRNN_SELF_QUERY 0x1u  /* queries are the grid's own points, same order;
                                 reference j == i is excluded by index */
#define FRNN_PATH_AUTO 0x0u   /* library (autotuner) chooses the path */
#define FRNN_PATH_GRID 0x2u   /* uniform-grid scan with the exact screen */
#define FRNN_PATH_TC 0x4u     /* tensor-core BF16 pre-filter + exact recheck
                                 (D >= 8 only) */

typedef struct frnn_ctx frnn_ctx;
typedef struct frnn_grid frnn_grid;

/* Library version as "major.minor.patch"; static storage. */
const char* frnn_version(void);

/*
 * Create a context on the current CUDA device.  The context owns the reused,
 * pre-allocated device workspace of Sec. 4.1 (all intermediate buffers of a
 * search live in it, so a repeated search allocates nothing) and keeps
 * inputs and outputs device-resident.
 *   cuda_stream       cudaStream_t to enqueue on (NULL = the legacy default
 *                     stream).  Not owned.
 *   mem_budget_bytes  cap on device memory the context may hold for grids and
 *                     workspace (0 = no cap).  Requests beyond it fail with
 *                     FRNN_ERR_BUDGET.
 * On success *out receives the context.  Errors: INVALID_ARG (out NULL),
 * CUDA (no usable device), OUT_OF_MEMORY.
 */
frnn_status frnn_create(frnn_ctx** out, void* cuda_stream, size_t mem_budget_bytes);

/* Release the workspace of frnn_create (Sec. 4.1).
 * Synchronise the context's stream and free everything it owns.  Grids built
 * through it are detached: they can no longer be queried, and must still be
 * released with frnn_grid_destroy.  NULL is accepted. */
frnn_status frnn_destroy(frnn_ctx* ctx);

/*
 * Build the uniform grid over reference points (Sec. 2: the uniform-grid /
 * cell-list method of the original FRNN, whose spacing divides r; Table 1
 * "roundoff-safe grid").
 *   refs  device, [N, D] row-major float32.  Read during the call's device
 *         work only; the grid keeps its own cell-sorted copy.
 *   N     number of points (>= 0)
 *   D     dimensions, 1..16
 *   r     the largest radius this grid will be queried with
 *   grid  in/out.  If *grid is NULL a new grid is allocated.  If *grid is a
 *         grid from this context with D equal and capacity >= N, it is rebuilt
 *         in place without allocating (the previous contents are replaced).
 * The grid bins at most 5 coordinates (by default up to D = 8 the last
 * min(D, 5), or the last 4 when the cell budget would make five-axis cells
 * too coarse; from D = 9 the last 4; see FRNN_OPT_GRID_NAXES and
 * FRNN_OPT_GRID_AXES) with cells of edge (r/m)(1+2^-10), m = the
 * cell-multiple option, enlarged when needed so that the cell count stays
 * bounded; the choice never changes results (the cell assignment is proven
 * conservative).  A non-finite coordinate makes frnn_sync return
 * FRNN_ERR_NONFINITE and later queries on the grid return no neighbours.
 */
frnn_status frnn_build_grid(frnn_ctx* ctx, const float* refs, int64_t N, int D, float r,
                            frnn_grid** grid);

/* Parameters a built grid received (the build derives them on the device
 * from the points' bounding box; none of them changes results).
 * Synchronises the grid's context stream.  Errors: INVALID_ARG (NULL
 * argument or a detached grid), CUDA. */
typedef struct frnn_grid_info {
    int naxes;          /* gridded coordinates (1..5) */
    int cell_mult;      /* m: the scan reaches +-m cells per gridded axis */
    int axes[5];        /* gridded coordinate indices (the first naxes) */
    int dims[5];        /* cells per gridded axis */
    float cell_edge;    /* 1 / inv_h, the cell edge (about r / m) */
    int64_t cells;      /* product of dims */
    int kernel;         /* grid scan used for this grid: 0 chunks of 16 queries
                           (candidates on lanes), 1 row tasks of 16 queries
                           (grids requested with up to four axes) */
    int valid;          /* 0 if a coordinate was non-finite */
} frnn_grid_info;

frnn_status frnn_grid_params(const frnn_grid* grid, frnn_grid_info* info);

/* Free a grid (after its pending work completes).  NULL is accepted.  A grid
 * is the device-resident cell structure of Sec. 2's uniform-grid method; it
 * stays resident between queries until this call. */
frnn_status frnn_grid_destroy(frnn_grid* grid);

/*
 * Fixed-radius query (Eq. 1) of M points against a grid.
 *   queries  device, [M, D] row-major float32.  With FRNN_SELF_QUERY it must
 *            be the pointer the grid was built from, and M its N.
 *   r        radius, 0 < r <= the grid's r
 *   K        neighbours kept per query, 1..1024
 *   flags    FRNN_SELF_QUERY | one FRNN_PATH_*
 *   counts   device, [M] int32 out: min(degree, K)
 *   idx      device, [M, K] int32 out: original reference indices
 *   dist2    device, [M, K] float32 out: squared distances (the contract's s)
 * Rows follow the original query order.  Errors: INVALID_ARG, UNSUPPORTED
 * (FRNN_PATH_TC with D < 8), BUDGET, OUT_OF_MEMORY, CUDA.
 */
frnn_status frnn_query(frnn_ctx* ctx, const frnn_grid* grid, const float* queries, int64_t M,
                       float r, int K, unsigned flags, int32_t* counts, int32_t* idx,
                       float* dist2);

/* One independent event of a batched call: a self-query of pts. */
typedef struct frnn_event {
    const float* pts; /* device, [n, D] row-major float32 */
    int64_t n;        /* points in this event (>= 0) */
    int32_t* counts;  /* device, [n] out */
    int32_t* idx;     /* device, [n, K] out */
    float* dist2;     /* device, [n, K] out */
} frnn_event;

/*
 * Self-query of many independent events of uneven size.  The paper evaluates
 * one tracking event at a time (Sec. 4.1) and has no batched interface: this
 * call applies Eq. 1 to every event of a batch, with the same result as one
 * call per event.  Each event is its own point set; no pair crosses events.
 * All events' grids are built by one set
 * of segmented launches and all queries run in one persistent launch, the
 * whole sequence captured once in a CUDA graph and replayed while the event
 * list (pointers and sizes) stays the same.  Results per event are bit-identical
 * to frnn_build_grid + frnn_query(FRNN_SELF_QUERY) on that event alone.
 *   ev        host array of n_events descriptors (copied; device buffers are
 *             the caller's)
 *   flags     FRNN_SELF_QUERY is implied; FRNN_PATH_* as for frnn_query
 * Errors: INVALID_ARG, BUDGET, OUT_OF_MEMORY, CUDA.
 */
frnn_status frnn_query_batched(frnn_ctx* ctx, const frnn_event* ev, int n_events, int D,
                               float r, int K, unsigned flags);

/*
 * The whole path with HOST buffers: copies refs to the device, builds the
 * grid, self-queries it and copies the results back, synchronising before it
 * returns (the host-side interface of Sec. 4.2's NumPy binding comparison).
 * Host buffers may be pageable.  When all three output buffers are
 * page-locked (cudaHostAlloc / cudaHostRegister), the query kernels write the
 * rows straight into them over the host link instead of staging them in
 * device memory and copying them back.
 *   refs_host [N, D] float32 in; counts_host [N], idx_host [N, K],
 *   dist2_host [N, K] out.  Device memory is taken from the context's
 *   workspace and reused across calls.
 */
frnn_status frnn_self_query_host(frnn_ctx* ctx, const float* refs_host, int64_t N, int D,
                                 float r, int K, unsigned flags, int32_t* counts_host,
                                 int32_t* idx_host, float* dist2_host);

/*
 * Serving loop with continuous batching.  Requests (independent events, host
 * buffers) arrive at the given times; whenever one of n_slots device streams
 * is free, the requests that have arrived are admitted in arrival order as
 * one batch, as many as fit max_batch and the device bytes still free under
 * mem_budget_bytes (0 = no cap; per request: input, outputs, its grid and
 * operands, estimated from n, D and K).  Each batch is copied in, built and
 * queried as one frnn_query_batched call and copied back on its own stream,
 * overlapping with the batches still running; its grids stay resident until
 * it completes.  Results are bit-identical to single-event queries.  Runs
 * until every request completed (synchronous; real time, so arrival_s values
 * pace the run).  A request larger than the whole budget is not run
 * (latency -1) and the call returns FRNN_ERR_BUDGET after serving the rest.
 * With n_slots = 1 and max_batch = 1 the loop serves one event at a time
 * (the sequential baseline).
 */
typedef struct frnn_request {
    const float* pts; /* host [n, D] float32 (page-locked memory copies faster) */
    int64_t n;
    int32_t* counts;  /* host [n] out */
    int32_t* idx;     /* host [n, K] out */
    float* dist2;     /* host [n, K] out */
    double arrival_s; /* arrival time, seconds after the call starts (>= 0) */
} frnn_request;

typedef struct frnn_serve_stats {
    double wall_s;                  /* first arrival to last completion */
    double p50_ms, p99_ms, mean_ms, max_ms;   /* arrival -> results in host memory */
    double events_per_s;            /* completed requests / wall_s */
    int64_t completed, rejected;
    int64_t peak_inflight_bytes;    /* estimated device bytes admitted at once */
    int peak_inflight_batches;      /* batches on the device at once */
} frnn_serve_stats;

frnn_status frnn_serve_run(frnn_ctx* ctx, const frnn_request* reqs, int n_reqs, int D, float r,
                           int K, size_t mem_budget_bytes, int n_slots, int max_batch,
                           double* latency_ms, frnn_serve_stats* stats);

/*
 * Self-query that allocates nothing (the paper has no counterpart: it is an
 * addition for callers that cannot allocate memory when they query).  Some
 * callers cannot call cudaMalloc or any allocating routine at query time:
 * a host loop that runs under a fixed, pre-reserved memory plan (embedded or
 * real-time code, or a process that divides device memory among several
 * engines in advance), or code that runs where an allocation is not allowed
 * or would synchronise the device.  This call needs no context: the grid, the
 * counters and the status word live in one fixed array of device memory
 * (about 7 MB) that the library declares statically; every GPU that loads
 * the library keeps that array until the process exits.
 *   pts      device, [N, D] row-major float32; N <= 65536 (larger N returns
 *            FRNN_ERR_INVALID_ARG at once), 1 <= D <= 16
 *   r, K     as for frnn_query (grid path, self-query, reference j == i
 *            excluded by index)
 *   counts, idx, dist2   device outputs as for frnn_query
 *   cuda_stream          stream to run on (NULL = legacy default stream)
 * Synchronous: it waits for its work and returns the device status
 * (FRNN_ERR_NONFINITE for a NaN or infinite coordinate).  Results are
 * bit-identical to frnn_build_grid + frnn_query(FRNN_SELF_QUERY).
 * Every call shares the one array and leaves its contents there (each call
 * clears what must start at zero); calls whose work overlaps on the GPU
 * (other streams or host threads) race on it and must be serialised by the
 * caller.  Each call looks the array's device address up with the caller's
 * device current.  The first call on a device also loads the library's
 * device code there, which places the array: make that first call before
 * any stream capture begins.  Error paths may allocate host memory for
 * their message; the query itself allocates nothing.
 */
frnn_status frnn_self_query_noalloc(const float* pts, int64_t N, int D, float r, int K,
                                    int32_t* counts, int32_t* idx, float* dist2,
                                    void* cuda_stream);

/* Wait for the context's stream and report (then clear) the device status
 * word: FRNN_OK or the first device-side error since the last sync.  The
 * paper specifies no error interface; this call exists because the work is
 * asynchronous (device-resident input and output, Sec. 4.1) and device-side
 * conditions can only be read back after it. */
frnn_status frnn_sync(frnn_ctx* ctx);

/* Text of the last error on this context (static storage of the context;
 * "" when none).  ctx NULL gives the last frnn_create failure. */
const char* frnn_last_error(const frnn_ctx* ctx);

/*
 * Autotuner.  Times the candidate configurations on the given point set (a
 * representative event, device memory, self-query): the automatic axis
 * choice with cell multiple m = 1 (five coordinates, or four when the cell
 * budget makes five-axis cells too coarse; scanned by chunks of 16 queries,
 * candidates on lanes, either candidate staging), four coordinates with
 * m = 1 and three with m = 2 (scanned by 16-query row tasks, at the default
 * and a later warp vote); fewer axes when D is smaller; for D <= 4 the
 * automatic choice with m = 2 as well, and for D <= 3 with m = 3 (where
 * the chunk scan's 128-row neighbour table holds the (2m + 1)^(axes - 1)
 * rows); on each grid, the tensor-core pre-filter (D >= 8).
 * Each candidate runs whole steps, build then query (first run untimed,
 * best of three timed with CUDA events on the context's stream, the L2
 * cache flushed before each run), and the fastest is cached for the event
 * size class (power-of-two bucket of N, D,
 * power-of-two bucket of K).  Afterwards FRNN_PATH_AUTO queries, grid builds
 * with the cell-multiple option at 0 (the default) and every event of
 * frnn_query_batched use the cached choice of their size class.  Results
 * never depend on the choice.  flags: FRNN_PATH_GRID or FRNN_PATH_TC limits
 * the candidates to that path (0: all).  Synchronises; allocates temporary
 * outputs (N + 2 N K words) and a flush buffer of twice the L2 size.  best
 * (may be NULL) receives the winner.
 */
typedef struct frnn_tune_result {
    int path;        /* FRNN_PATH_GRID or FRNN_PATH_TC */
    int cell_mult;   /* m */
    int exit_dims;   /* warp vote point of the row-task scan (0 = default) */
    float ms;        /* build + query time of the winner, milliseconds */
    int grid_axes;   /* gridded coordinates requested (0: the automatic choice; 3 or 4) */
    int staging;     /* grid scan candidate staging (FRNN_OPT_STAGING values 1, 2) */
} frnn_tune_result;

frnn_status frnn_autotune(frnn_ctx* ctx, const float* refs, int64_t N, int D, float r, int K,
                          unsigned flags, frnn_tune_result* best);

/* Tunable options (none changes results, only speed). */
typedef enum frnn_option {
    FRNN_OPT_CELL_MULT = 1,   /* m in {1, 2, 3}: cell edge ~ r/m, search +-m cells;
                                 0 (default): autotuned, else 2 on grids of at
                                 most three requested axes and 1 otherwise */
    FRNN_OPT_GRID_AXES = 2,   /* which coordinates are gridded: 0 the last ones,
                                 1 the widest ones (count: FRNN_OPT_GRID_NAXES) */
    FRNN_OPT_EXIT_DIMS = 3,   /* row-task grid scan (grids of up to four axes):
                                 dims summed before its warp-uniform early
                                 exit (0 = library default); the chunk scan of
                                 five-axis grids ignores it */
    FRNN_OPT_USE_GRAPH = 4,   /* 1 (default): batched calls replay a CUDA graph */
    FRNN_OPT_AUTOTUNE = 5,    /* 1 (default): FRNN_PATH_AUTO consults the tuner;
                                 setting 0 also clears the tuned cache */
    FRNN_OPT_AUTO_TC = 6,     /* 1 (default): FRNN_PATH_AUTO takes the tensor-core
                                 path for D >= 8 */
    FRNN_OPT_TC_SURVIVORS = 7,/* read: candidates that passed the tensor-core
                                 pre-filter since the last reset (synchronises);
                                 set (any value): reset both counters */
    FRNN_OPT_TC_ACCEPTED = 8, /* read: of those, accepted by the exact recheck */
    FRNN_OPT_KERNEL_TIMING = 9,/* 1: frnn_query records CUDA events around its
                                 main query kernel (grid or tensor-core; not the
                                 selection pass or operand preparation), read
                                 with frnn_kernel_times; 0 (default): off.
                                 Setting it discards recorded pairs. */
    FRNN_OPT_GRID_NAXES = 10, /* gridded coordinates: 1..5 (at most D); 0
                                 (default): autotuned, else up to D = 8 the
                                 build's choice between min(D, 5) and one
                                 fewer (the smaller expected neighbourhood
                                 under the cell budget), from D = 9 four.
                                 Grids requested with 1..4 axes are scanned by
                                 16-query row tasks, five-axis and automatic
                                 ones by 16-query chunks.  The cell multiple
                                 is lowered until the neighbour rows,
                                 (2m+1)^(axes-1), are at most 32 (row tasks)
                                 or 128 (chunks). */
    FRNN_OPT_STAGING = 11     /* candidate staging of the grid scan: 1 each lane
                                 loads its candidate's row from global memory
                                 (L2), the next round in flight; 2 bulk copies
                                 (cp.async.bulk) of tiles into a shared-memory
                                 ring; 0 (default): autotuned, else 1 */
} frnn_option;

frnn_status frnn_set_option(frnn_ctx* ctx, frnn_option opt, int64_t value);
frnn_status frnn_get_option(const frnn_ctx* ctx, frnn_option opt, int64_t* value);

/* Compact output, first pass: count-first exact allocation (Sec. 4: the
 * temporary edge capacity of the real event fell from 4.35 GB to 148 MB; the
 * compact output is one of the retained ideas of Sec. 6).  Runs the search of
 * frnn_query (same arguments, same path choice, same results) once, keeps the
 * sorted rows in the context, and writes
 *   offsets  device int64 [M + 1]: row i's entries will occupy
 *            [offsets[i], offsets[i+1]) of the fill pass's arrays;
 *            offsets[i+1] - offsets[i] = min(degree_i, K); offsets[0] = 0
 *   degree   device int32 [M] or NULL: the full number of in-radius
 *            neighbours of each query (not truncated to K; saturates at
 *            INT32_MAX), self excluded as in frnn_query
 *   n_edges  host out: offsets[M], the entries the caller must allocate.
 * Synchronises the context's stream (the count has to reach the host).  The
 * context holds 8 * 32 + 4 bytes of staging per query, reused
 * across calls (charged to the memory budget).  Errors: those of frnn_query
 * (INVALID_ARG, UNSUPPORTED, BUDGET, OUT_OF_MEMORY, NONFINITE, CAPACITY,
 * TIMEOUT, CUDA); NULL offsets or n_edges: INVALID_ARG. */
frnn_status frnn_query_csr_count(frnn_ctx* ctx, const frnn_grid* grid, const float* queries,
                                 int64_t M, float r, int K, unsigned flags, int64_t* offsets,
                                 int32_t* degree, int64_t* n_edges);

/* Compact output, second pass: writes the rows of the last
 * frnn_query_csr_count on this context into
 *   idx    device int32 [n_edges]: original reference indices, each row
 *          sorted by (d2, index) ascending as in frnn_query, no padding
 *   dist2  device float [n_edges]: the matching squared distances (bit-exact
 *          float32 contract, Eq. 1)
 * using the offsets array given to the count pass (still owned by the
 * caller and unchanged).  Asynchronous on the context's stream.  Any other
 * call on the context between the two passes (query, build, batched,
 * host-buffer, autotune, grid destroy) discards the pending rows: then, or
 * without a count pass, INVALID_ARG.  idx/dist2 may be NULL when n_edges was 0.
 * The paper's interface has no separate fill call; the split lets the caller
 * allocate exactly n_edges entries in between. */
frnn_status frnn_query_csr_fill(frnn_ctx* ctx, int32_t* idx, float* dist2);

/*
 * The whole path with HOST buffers and compact output, in one call: copies
 * refs to the device, builds the grid, runs the count pass of
 * frnn_query_csr_count (self-query) and, if the rows fit, the fill pass, then
 * copies the rows back; synchronises before it returns.  The fill's gather
 * starts before the edge count reaches the host, into device rows sized for
 * min(edge_cap, N K) entries (when those take at most 1 GiB; else it waits
 * for the count and is sized by it).  This is the shape of the paper's NumPy
 * binding (Sec. 4.2: host transfers and compact host output).
 *   refs_host     [N, D] float32 in
 *   offsets_host  [N + 1] int64 out: row i at [offsets[i], offsets[i+1])
 *   idx_host, dist2_host  [edge_cap] out (may be NULL when edge_cap is 0)
 *   edge_cap      entries the caller provided; N * min(K, degree bound) or
 *                 N * K always suffices
 *   n_edges       out: offsets[N], the number of entries
 * If n_edges > edge_cap the offsets are still written but no row is copied
 * and the call returns FRNN_ERR_CAPACITY (retry with a larger buffer).
 * Other errors: those of frnn_self_query_host.
 */
frnn_status frnn_self_query_host_csr(frnn_ctx* ctx, const float* refs_host, int64_t N, int D,
                                     float r, int K, unsigned flags, int64_t* offsets_host,
                                     int32_t* idx_host, float* dist2_host, int64_t edge_cap,
                                     int64_t* n_edges);

/* Check of the device-side failure handling (no counterpart in the paper).
 * Launches one warp on the context's stream that waits on an mbarrier which
 * nothing ever completes, with the bounded wait every query kernel uses but a
 * limit of limit_ns nanoseconds of %globaltimer time (1e6 .. 5e9).  The wait
 * runs out, the warp records a timeout in the context's status word and
 * exits; the call then synchronises and returns what frnn_sync returns:
 * FRNN_ERR_TIMEOUT when the bound works.  The status word is cleared, so the
 * context stays usable.  Errors: INVALID_ARG (NULL ctx, limit out of range),
 * CUDA. */
frnn_status frnn_check_wait_timeout(frnn_ctx* ctx, uint64_t limit_ns);

/* Durations of the main query kernel of every frnn_query call made since the
 * last frnn_kernel_times call (or since FRNN_OPT_KERNEL_TIMING was set), in
 * milliseconds, in call order.  Synchronises the context's stream.
 *   ms    host array of `max` floats (may be NULL when max == 0)
 *   n     out: number of durations recorded (may exceed max; only the first
 *         max are written)
 * Up to 4096 calls are recorded between reads; later calls are not timed.
 * Clears the record.  The queries that frnn_self_query_host and the
 * autotuner's trials make through frnn_query are recorded too; batched and
 * serving calls record nothing.
 * The paper reports kernel times but specifies no such interface; this is
 * measurement plumbing.  Errors: INVALID_ARG (NULL ctx or n, max < 0, ms NULL
 * with max > 0), CUDA. */
frnn_status frnn_kernel_times(frnn_ctx* ctx, float* ms, int max, int* n);

#ifdef __cplusplus
}
#endif

#endif /* FRNN_H */
