// api.cu — the C ABI (include/frnn.h): contexts, grids, argument validation,
// the single-event, cross-set, batched (CUDA-graph) and host-buffer paths.
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <unordered_set>
#include <vector>

#include "frnn_host.h"

using namespace frnn;

struct frnn_grid {
    frnn_ctx* ctx = nullptr;
    GridBufs g;
    const float* refs = nullptr;
    int64_t N = 0;
    int D = 0;
    float r = 0.f;
    int naxes = 0;   // gridded axes requested at the build
};

struct frnn_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;        // 0 = no cap
    size_t held = 0;          // bytes of grids + workspaces currently held
    int32_t* d_status = nullptr;
    int32_t* h_status = nullptr;
    unsigned long long* d_tcstat = nullptr;   // [2] tensor-core survivors / exact accepts
    std::string err;
    // options (cell_mult 0 / exit_dims 0: tuned value, else the library default)
    int cell_mult = 0;
    int grid_naxes = 0;       // gridded axes: 0 tuned / default, else 1..4
    int axes_mode = 0;
    int exit_dims = 0;
    int staging = 0;          // FRNN_OPT_STAGING (0: tuned, else 1)
    int use_graph = 1;
    int autotune = 1;
    int auto_tc = 1;          // FRNN_PATH_AUTO uses the tensor-core path for D >= 8
    // workspaces
    GridBufs qset;            // cross-set query binning
    GridBufs batch;           // batched multi-event grid
    frnn_grid* host_grid = nullptr;   // grid of the host-buffer path
    void* hp_buf = nullptr;   // device buffers of the host-buffer path
    size_t hp_bytes = 0;
    void* hr_buf = nullptr;   // compact rows of the host-buffer path
    size_t hr_bytes = 0;
    // autotuner cache: (log2 N bucket, D, log2 K bucket) -> best configuration
    struct Tuned {
        int path;    // 0 grid, 1 tensor-core
        int m;
        int exit_dims;
        float ms;
        int naxes;
        int staging;   // FRNN_OPT_STAGING value (1 or 2)
    };
    std::map<uint32_t, Tuned> tuned;
    // live grids built through this context (detached when it is destroyed)
    std::unordered_set<frnn_grid*> grids;
    // batched graph cache; captured and replayed on an internal stream fenced
    // to the context's stream with events (the legacy default stream cannot
    // be captured)
    cudaStream_t gstream = nullptr;
    cudaEvent_t g_in = nullptr, g_out = nullptr;
    cudaEvent_t ev_edges = nullptr;   // host-buffer compact path: edge count copied back
    // host-buffer compact path: a copy stream for the rows, and one event per
    // part of the gather plus one for the finished copies
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_part[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_copied = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<frnn_event> g_ev;
    int g_D = 0, g_K = 0;
    float g_r = 0.f;
    unsigned g_flags = 0;
    int g_opts[5] = {0, 0, 0, 0, 0};
    // compact output: staging rows of the pending count pass, and what the
    // fill pass needs (valid until the next call on this context)
    void* csr_buf = nullptr;
    size_t csr_bytes = 0;
    int32_t* csr_cnt = nullptr;     // [M] marked counts, original order
    int32_t* csr_idx = nullptr;     // [M * kCsrStageW] staged rows
    float* csr_d2 = nullptr;
    int64_t* csr_parts = nullptr;
    bool csr_pending = false;
    QueryLaunch csr_q{};
    int64_t csr_M = 0, csr_E = 0;
    const int64_t* csr_off = nullptr;
    // kernel timing (FRNN_OPT_KERNEL_TIMING): event pairs, reused across reads
    int ktime = 0;
    std::vector<cudaEvent_t> kev;   // 2 per recorded call
    int kev_used = 0;               // pairs recorded since the last read
};

static constexpr int kMaxTimedCalls = 4096;

static thread_local std::string g_create_err;

namespace frnn {
void ctx_copy_tuning(frnn_ctx* dst, const frnn_ctx* src) {
    dst->cell_mult = src->cell_mult;
    dst->grid_naxes = src->grid_naxes;
    dst->axes_mode = src->axes_mode;
    dst->exit_dims = src->exit_dims;
    dst->staging = src->staging;
    dst->autotune = src->autotune;
    dst->auto_tc = src->auto_tc;
    dst->tuned = src->tuned;
}
void ctx_set_error(frnn_ctx* ctx, const char* msg) {
    if (ctx) ctx->err = msg;
}
}  // namespace frnn

static int grid_kernel(int naxes);

static frnn_status fail(frnn_ctx* c, frnn_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

static frnn_status cuda_fail(frnn_ctx* c, cudaError_t e, const char* what) {
    cudaGetLastError();
    return fail(c, FRNN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Device address of a page-locked host buffer (NULL if the buffer is pageable
// or unknown to CUDA).  On a Grace-Blackwell node such memory is reachable
// from the GPU over the coherent chip-to-chip link, so kernels can write
// results straight into it instead of staging them in HBM and copying.
namespace frnn {
void* mapped_host(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}
}  // namespace frnn

static bool radius_ok(float r) {
    return std::isfinite(r) && r >= 0x1p-60f && r <= 0x1p60f;
}

static bool budget_allows(frnn_ctx* c, size_t old_bytes, size_t new_bytes) {
    if (c->budget == 0) return true;
    return c->held - old_bytes + new_bytes <= c->budget;
}

// Predicted device bytes of a GridBufs layout (mirrors grid_alloc's layout).
static size_t predict_grid_bytes(int E, const int64_t* n, int D, const int64_t* caps) {
    const int DP = padded_dim(D);
    int64_t nt = 0, L = 0;
    for (int e = 0; e < E; ++e) {
        nt += n[e] + 1;
        L += caps[e] + 1;
    }
    nt = std::max<int64_t>(nt, 1);
    size_t b = 0;
    b += sizeof(EventHdr) * E + 16 * (E + 1) + sizeof(int32_t) * kBBoxStride * kBBoxCopies * E;
    b += (size_t)(nt + kTcRowPad) * sizeof(float) * DP +
         (size_t)nt * (4 * sizeof(int32_t) + sizeof(Overflow));
    b += (size_t)L * sizeof(int32_t) + (size_t)(L / 2048 + 1) * sizeof(int32_t);
    b += 64 * 1024 + 16 * 256;
    return b;
}

static int build_naxes(const frnn_ctx* ctx, int64_t N, int D);
// gridded axes a cell budget is sized for: the requested count, or for the
// automatic choice (0) the most the build may take
static int cap_axes(int naxes, int D) { return naxes > 0 ? naxes : std::min(D, kMaxAxes); }

static frnn_status alloc_accounted(frnn_ctx* c, GridBufs& g, int E, const int64_t* n, int D,
                                   const int64_t* caps_in) {
    std::vector<int64_t> caps(E);
    for (int e = 0; e < E; ++e)
        caps[e] = caps_in ? caps_in[e] : cell_cap_for(n[e], cap_axes(build_naxes(c, n[e], D), D));
    const size_t old_bytes = g.bytes;
    const size_t need = predict_grid_bytes(E, n, D, caps.data());
    const bool reuse = g.base && need <= g.bytes;
    if (!reuse && !budget_allows(c, old_bytes, need))
        return fail(c, FRNN_ERR_BUDGET, "request exceeds the context's memory budget");
    std::string err;
    frnn_status s = grid_alloc(g, E, n, D, err, caps.data());
    c->held = c->held - old_bytes + g.bytes;
    if (s != FRNN_OK) return fail(c, s, err);
    return FRNN_OK;
}

// Path choice: FRNN_PATH_TC forces the tensor-core pre-filter (D >= 8),
// FRNN_PATH_GRID the scalar grid scan; FRNN_PATH_AUTO takes the tensor-core
// path for D >= 8 unless the context's option says otherwise.
static bool default_tc(const frnn_ctx* ctx, int D, int naxes);
static const frnn_ctx::Tuned* find_tuned(const frnn_ctx* ctx, int64_t N, int D, int K);
// naxes: gridded axes of the grid being queried (-1: what a build would use now)
static bool use_tc_path(const frnn_ctx* ctx, int D, unsigned flags, int64_t N = -1, int K = -1,
                        int naxes = -1) {
    if (flags & FRNN_PATH_TC) return true;
    if (flags & FRNN_PATH_GRID) return false;
    if (D < 8) return false;
    if (N >= 0) {
        const frnn_ctx::Tuned* t = find_tuned(ctx, N, D, K);
        if (t) return t->path == 1;
    }
    return default_tc(ctx, D, naxes >= 0 ? naxes : build_naxes(ctx, std::max<int64_t>(N, 0), D));
}

// Build (or reuse) the tensor-core operands of a point set; accounted in the
// context's memory budget.
namespace frnn {
frnn_status ctx_reserve_batch(frnn_ctx* ctx, int E, int64_t n, int D, int K, unsigned flags) {
    if (E < 1 || n < 1) return FRNN_OK;
    std::vector<int64_t> ns(E, n);
    frnn_status s = alloc_accounted(ctx, ctx->batch, E, ns.data(), D, nullptr);
    if (s != FRNN_OK || !use_tc_path(ctx, D, flags, n, K)) return s;
    std::string err;
    s = tc_reserve(ctx->batch, err);
    return s == FRNN_OK ? s : fail(ctx, s, err);
}
}  // namespace frnn

static frnn_status prepare_tc(frnn_ctx* ctx, GridBufs& g, const GridBufs& center_src,
                              bool capturing = false) {
    if (g.tc_ready && &g == &center_src) return FRNN_OK;
    const size_t before = g.tc_bytes;
    std::string err;
    frnn_status s = tc_prepare(g, center_src, ctx->d_status, capturing ? ctx->gstream : ctx->stream,
                               err);
    ctx->held = ctx->held - std::min(ctx->held, before) + g.tc_bytes;
    if (s != FRNN_OK) return fail(ctx, s, err);
    return FRNN_OK;
}

// The grid scan for a grid requested with naxes gridded axes (0: the
// build's automatic choice, five or four): the row-task kernel for grids
// requested with up to four axes (cells holding many points, long candidate
// streams shared by 16 queries), the chunk kernel otherwise (few points per
// cell, candidates on lanes).
static int grid_kernel(int naxes) { return (naxes >= 1 && naxes <= 4) ? 1 : 0; }

// Pair copy and tasks of a point set for the row-task kernel; accounted in
// the context's memory budget.
static frnn_status prepare_rows(frnn_ctx* ctx, GridBufs& g, cudaStream_t st) {
    if (g.rows_ready) return FRNN_OK;
    const size_t before = g.rows_bytes;
    std::string err;
    frnn_status s = rows_prepare(g, ctx->d_status, st, err);
    ctx->held = ctx->held - std::min(ctx->held, before) + g.rows_bytes;
    if (s != FRNN_OK) return fail(ctx, s, err);
    return FRNN_OK;
}

static int log2_bucket(int64_t x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}
static uint32_t tune_key(int64_t N, int D, int K) {
    return (uint32_t)log2_bucket(N) | ((uint32_t)D << 8) | ((uint32_t)log2_bucket(K) << 16);
}
// Tuned entry for this size class; K < 0 matches any K (grid builds do not know K).
static const frnn_ctx::Tuned* find_tuned(const frnn_ctx* ctx, int64_t N, int D, int K) {
    if (!ctx->autotune) return nullptr;
    if (K >= 0) {
        auto it = ctx->tuned.find(tune_key(N, D, K));
        return it == ctx->tuned.end() ? nullptr : &it->second;
    }
    const uint32_t lo = (uint32_t)log2_bucket(N) | ((uint32_t)D << 8);
    for (auto& kv : ctx->tuned)
        if ((kv.first & 0xFFFFu) == lo) return &kv.second;
    return nullptr;
}
// cell multiple for a build: explicit option, else tuned, else 1
static int build_mult(const frnn_ctx* ctx, int64_t N, int D) {
    if (ctx->cell_mult > 0) return ctx->cell_mult;
    const frnn_ctx::Tuned* t = find_tuned(ctx, N, D, -1);
    if (t) return t->m;
    // default: cells of r/2 when at most three coordinates are gridded on
    // request (a finer grid pays there), cells of r otherwise
    const int na = build_naxes(ctx, N, D);
    return (na >= 1 && na <= 3 && D > 3) ? 2 : 1;
}
// gridded axes when neither the option nor the tuner fixes them.  Up to
// D = 8: 0, the build's automatic choice (five axes, or four when the cell
// budget makes five-axis cells too coarse; all of them for D < 5), scanned by
// the chunk kernel.  From D = 9: four axes, scanned by the row-task kernel,
// whose packed pre-screen costs less per candidate pair than the chunk
// kernel's whole contract as D grows (measured build + query: 300k x 8 event
// 0.306 ms five axes vs 0.318 ms four; 500k x 12 event 0.639 vs 0.546 ms).
static int default_naxes(int D) { return D >= 9 ? 4 : 0; }
static int build_naxes(const frnn_ctx* ctx, int64_t N, int D) {
    if (ctx->grid_naxes > 0) return std::min(ctx->grid_naxes, D);
    const frnn_ctx::Tuned* t = find_tuned(ctx, N, D, -1);
    return std::min(t ? t->naxes : default_naxes(D), D);
}
// default path when nothing is tuned: the tensor-core pre-filter beats the
// grid scan over three gridded axes from about D = 10 on (0.90 vs 1.26 ms at
// 500k x 12), but not the scan over four (0.70 ms): its 128-query tasks are
// poorly filled by the shorter rows of a four-axis grid
static bool default_tc(const frnn_ctx* ctx, int D, int naxes) {
    return ctx->auto_tc && D >= 10 && naxes >= 1 && naxes <= 3;
}

extern "C" {

const char* frnn_version(void) { return "0.1.0"; }

frnn_status frnn_create(frnn_ctx** out, void* cuda_stream, size_t mem_budget_bytes) {
    if (!out) {
        g_create_err = "out is NULL";
        return FRNN_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_err = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return FRNN_ERR_CUDA;
    }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_err = std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e);
        return FRNN_ERR_CUDA;
    }
    if (prop.major < 10) {
        g_create_err = "this library is built for sm_103a (GB300); device is sm_" +
                       std::to_string(prop.major) + std::to_string(prop.minor);
        return FRNN_ERR_UNSUPPORTED;
    }
    frnn_ctx* c = new frnn_ctx();
    c->device = dev;
    c->num_sms = prop.multiProcessorCount;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->budget = mem_budget_bytes;
    if (cudaMalloc(&c->d_status, 64) != cudaSuccess ||
        cudaMallocHost(&c->h_status, 64) != cudaSuccess) {
        cudaGetLastError();
        g_create_err = "allocation of the status word failed";
        if (c->d_status) cudaFree(c->d_status);
        delete c;
        return FRNN_ERR_OUT_OF_MEMORY;
    }
    cudaMemsetAsync(c->d_status, 0, 64, c->stream);
    c->d_tcstat = reinterpret_cast<unsigned long long*>(c->d_status + 8);   // same block
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_err = std::string("stream unusable: ") + cudaGetErrorString(e);
        cudaFree(c->d_status);
        cudaFreeHost(c->h_status);
        delete c;
        return FRNN_ERR_CUDA;
    }
    *out = c;
    return FRNN_OK;
}

frnn_status frnn_grid_params(const frnn_grid* grid, frnn_grid_info* info) {
    if (!grid || !info || !grid->ctx) return FRNN_ERR_INVALID_ARG;
    frnn_ctx* ctx = grid->ctx;
    *info = frnn_grid_info{};
    info->kernel = grid_kernel(grid->naxes);
    if (grid->g.E < 1 || !grid->g.hdr) return FRNN_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    EventHdr h{};
    if (e == cudaSuccess) e = cudaMemcpy(&h, grid->g.hdr, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the grid header");
    info->naxes = h.naxes;
    info->cell_mult = h.m;
    info->cells = 1;
    for (int a = 0; a < kMaxAxes; ++a) {
        info->axes[a] = a < h.naxes ? h.axes[a] : 0;
        info->dims[a] = h.dims[a];
        info->cells *= h.dims[a];
    }
    info->cell_edge = h.inv_h > 0.f ? 1.f / h.inv_h : INFINITY;
    info->valid = h.valid;
    return FRNN_OK;
}

frnn_status frnn_grid_destroy(frnn_grid* grid) {
    if (!grid) return FRNN_OK;
    if (grid->ctx) {
        cudaStreamSynchronize(grid->ctx->stream);
        grid->ctx->csr_pending = false;
        grid->ctx->held -= std::min(grid->ctx->held,
                                    grid->g.bytes + grid->g.tc_bytes + grid->g.rows_bytes);
        grid->ctx->grids.erase(grid);
    } else {
        cudaDeviceSynchronize();   // context gone: its stream may still hold work on the buffers
    }
    grid_free(grid->g);
    delete grid;
    return FRNN_OK;
}

// The host-buffer paths keep one grid in the context; a call of another
// dimension cannot rebuild it in place (frnn_build_grid would make a new grid
// and drop this one), so it is released first.
static void release_host_grid_if_other_dim(frnn_ctx* ctx, int D) {
    if (ctx->host_grid && ctx->host_grid->D != D) {
        frnn_grid_destroy(ctx->host_grid);
        ctx->host_grid = nullptr;
    }
}

frnn_status frnn_destroy(frnn_ctx* ctx) {
    if (!ctx) return FRNN_OK;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->gstream) cudaStreamSynchronize(ctx->gstream);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    if (ctx->g_in) cudaEventDestroy(ctx->g_in);
    if (ctx->g_out) cudaEventDestroy(ctx->g_out);
    if (ctx->ev_edges) cudaEventDestroy(ctx->ev_edges);
    if (ctx->cstream) {
        cudaStreamSynchronize(ctx->cstream);
        cudaStreamDestroy(ctx->cstream);
    }
    for (cudaEvent_t ev : ctx->ev_part)
        if (ev) cudaEventDestroy(ev);
    if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
    for (cudaEvent_t e : ctx->kev) cudaEventDestroy(e);
    if (ctx->host_grid) {
        frnn_grid* g = ctx->host_grid;
        ctx->host_grid = nullptr;
        ctx->grids.erase(g);
        g->ctx = nullptr;
        grid_free(g->g);
        delete g;
    }
    // grids the caller still holds stay valid for frnn_grid_destroy only
    for (frnn_grid* g : ctx->grids) g->ctx = nullptr;
    ctx->grids.clear();
    grid_free(ctx->qset);
    grid_free(ctx->batch);
    if (ctx->hp_buf) cudaFree(ctx->hp_buf);
    if (ctx->hr_buf) cudaFree(ctx->hr_buf);
    if (ctx->csr_buf) cudaFree(ctx->csr_buf);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    delete ctx;
    return FRNN_OK;
}

frnn_status frnn_build_grid(frnn_ctx* ctx, const float* refs, int64_t N, int D, float r,
                            frnn_grid** grid) {
    if (ctx) ctx->csr_pending = false;
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    if (!grid) return fail(ctx, FRNN_ERR_INVALID_ARG, "grid is NULL");
    if (D < 1 || D > kMaxD) return fail(ctx, FRNN_ERR_INVALID_ARG, "D must be in 1..16");
    if (N < 0 || N >= INT32_MAX) return fail(ctx, FRNN_ERR_INVALID_ARG, "N out of range");
    if (N > 0 && !refs) return fail(ctx, FRNN_ERR_INVALID_ARG, "refs is NULL");
    if (!radius_ok(r)) return fail(ctx, FRNN_ERR_INVALID_ARG, "r must be finite, 2^-60..2^60");
    frnn_grid* g = *grid;
    if (g && (g->ctx != ctx || g->D != D)) g = nullptr;   // not reusable: make a new one
    const bool fresh = (g == nullptr);
    if (fresh) {
        g = new frnn_grid();
        g->ctx = ctx;
        g->D = D;
        ctx->grids.insert(g);
    }
    frnn_status s = alloc_accounted(ctx, g->g, 1, &N, D, nullptr);
    if (s != FRNN_OK) {
        if (fresh) {
            ctx->held -= std::min(ctx->held, g->g.bytes);
            ctx->grids.erase(g);
            grid_free(g->g);
            delete g;
        }
        return s;
    }
    g->refs = refs;
    g->N = N;
    g->r = r;
    BuildOpts o;
    o.r = r;
    o.m = build_mult(ctx, N, D);
    o.naxes = build_naxes(ctx, N, D);
    o.axes_mode = ctx->axes_mode;
    g->naxes = o.naxes;
    std::string err;
    const float* ev_refs[1] = {refs};
    s = enqueue_build(g->g, ev_refs, o, nullptr, ctx->d_status, ctx->stream, false, err);
    if (s != FRNN_OK) {
        if (fresh) frnn_grid_destroy(g);
        return fail(ctx, s, err);
    }
    *grid = g;
    return FRNN_OK;
}

static frnn_status check_query_args(frnn_ctx* ctx, int64_t M, float r, int K, unsigned flags,
                                    const int32_t* counts, const int32_t* idx,
                                    const float* dist2) {
    if (M < 0 || M >= INT32_MAX) return fail(ctx, FRNN_ERR_INVALID_ARG, "M out of range");
    if (K < 1 || K > kMaxK) return fail(ctx, FRNN_ERR_INVALID_ARG, "K must be in 1..1024");
    if (!radius_ok(r)) return fail(ctx, FRNN_ERR_INVALID_ARG, "r must be finite, 2^-60..2^60");
    if (flags & ~(FRNN_SELF_QUERY | FRNN_PATH_GRID | FRNN_PATH_TC))
        return fail(ctx, FRNN_ERR_INVALID_ARG, "unknown flag bits");
    if ((flags & FRNN_PATH_GRID) && (flags & FRNN_PATH_TC))
        return fail(ctx, FRNN_ERR_INVALID_ARG, "choose one path");
    if (M > 0 && (!counts || !idx || !dist2))
        return fail(ctx, FRNN_ERR_INVALID_ARG, "output pointer is NULL");
    return FRNN_OK;
}

// The search of frnn_query; csr != NULL: compact output's first pass (rows
// to the staging area, counts marked, spilled rows counted and marked).
struct CsrPass {
    int32_t* degree;
};
static frnn_status query_impl(frnn_ctx* ctx, const frnn_grid* grid, const float* queries,
                              int64_t M, float r, int K, unsigned flags, int32_t* counts,
                              int32_t* idx, float* dist2, const CsrPass* csr,
                              QueryLaunch* launched) {
    frnn_status s;
    if (r > grid->r) return fail(ctx, FRNN_ERR_INVALID_ARG, "r exceeds the grid's radius");
    if (M > 0 && !queries) return fail(ctx, FRNN_ERR_INVALID_ARG, "queries is NULL");
    const bool self = (flags & FRNN_SELF_QUERY) != 0;
    if (self && (queries != grid->refs || M != grid->N))
        return fail(ctx, FRNN_ERR_INVALID_ARG,
                    "FRNN_SELF_QUERY needs the grid's own points (same pointer and count)");
    if ((flags & FRNN_PATH_TC) && grid->D < 8)
        return fail(ctx, FRNN_ERR_UNSUPPORTED, "the tensor-core path needs D >= 8");
    if (M == 0) return FRNN_OK;
    QueryLaunch q{};
    q.rset = &grid->g;
    q.r2 = r * r;
    q.K = K;
    q.self = self ? 1 : 0;
    q.exit_dims = ctx->exit_dims;
    {
        int stg = ctx->staging;
        const frnn_ctx::Tuned* t = find_tuned(ctx, grid->N, grid->D, K);
        if (stg == 0 && t) stg = t->staging;
        if (q.exit_dims == 0 && t && !(flags & (FRNN_PATH_GRID | FRNN_PATH_TC)))
            q.exit_dims = t->exit_dims;
        q.stage = stg == 2 ? 1 : 0;
    }
    q.counts = counts;
    q.idx = idx;
    q.dist2 = dist2;
    q.d_status = ctx->d_status;
    q.num_sms = ctx->num_sms;
    if (csr) {
        q.csr = 1;
        q.ovf_mode = 1;
        q.degree = csr->degree;
    }
    if (ctx->ktime && ctx->kev_used < kMaxTimedCalls) {
        const size_t need = 2 * (size_t)(ctx->kev_used + 1);
        while (ctx->kev.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            ctx->kev.push_back(e);
        }
        if (ctx->kev.size() >= need) {
            q.kev[0] = ctx->kev[need - 2];
            q.kev[1] = ctx->kev[need - 1];
            ++ctx->kev_used;
        }
    }
    std::string err;
    GridBufs& rg = const_cast<frnn_grid*>(grid)->g;   // tensor-core operands are a lazy cache
    if (self) {
        q.qset = &rg;
    } else {
        const int64_t cap = grid->g.h_hdr[0].cell_cap;
        s = alloc_accounted(ctx, ctx->qset, 1, &M, grid->D, &cap);
        if (s != FRNN_OK) return s;
        BuildOpts o;
        const float* ev_q[1] = {queries};
        s = enqueue_build(ctx->qset, ev_q, o, &grid->g, ctx->d_status, ctx->stream, false, err);
        if (s != FRNN_OK) return fail(ctx, s, err);
        q.qset = &ctx->qset;
    }
    if (use_tc_path(ctx, grid->D, flags, grid->N, K, grid->naxes)) {
        s = prepare_tc(ctx, rg, rg);
        if (s == FRNN_OK && !self) s = prepare_tc(ctx, ctx->qset, rg);
        if (s != FRNN_OK) return s;
        q.tc_stats = ctx->d_tcstat;
        s = enqueue_tc_query(q, ctx->stream, err);
    } else {
        q.kernel = grid_kernel(grid->naxes);
        if (q.kernel == 1) {
            s = prepare_rows(ctx, rg, ctx->stream);
            if (s == FRNN_OK && !self) s = prepare_rows(ctx, ctx->qset, ctx->stream);
            if (s != FRNN_OK) return s;
        }
        s = enqueue_grid_query(q, ctx->stream, err);
    }
    if (s != FRNN_OK) return fail(ctx, s, err);
    q.kev[0] = q.kev[1] = nullptr;
    if (launched) *launched = q;
    return FRNN_OK;
}

frnn_status frnn_query(frnn_ctx* ctx, const frnn_grid* grid, const float* queries, int64_t M,
                       float r, int K, unsigned flags, int32_t* counts, int32_t* idx,
                       float* dist2) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    ctx->csr_pending = false;
    if (!grid || grid->ctx != ctx) return fail(ctx, FRNN_ERR_INVALID_ARG, "grid is not of ctx");
    frnn_status s = check_query_args(ctx, M, r, K, flags, counts, idx, dist2);
    if (s != FRNN_OK) return s;
    return query_impl(ctx, grid, queries, M, r, K, flags, counts, idx, dist2, nullptr, nullptr);
}

static frnn_status csr_reserve(frnn_ctx* ctx, int64_t M) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t rows = (size_t)std::max<int64_t>(M, 1);
    const size_t b_cnt = al(rows * 4), b_stage = al(rows * kCsrStageW * 4);
    const size_t b_parts = al((size_t)csr_parts_needed(M) * 8);
    const size_t need = b_cnt + 2 * b_stage + b_parts;
    if (need > ctx->csr_bytes) {
        if (!budget_allows(ctx, ctx->csr_bytes, need))
            return fail(ctx, FRNN_ERR_BUDGET, "request exceeds the context's memory budget");
        cudaStreamSynchronize(ctx->stream);
        if (ctx->csr_buf) cudaFree(ctx->csr_buf);
        ctx->held -= ctx->csr_bytes;
        ctx->csr_buf = nullptr;
        ctx->csr_bytes = 0;
        if (cudaMalloc(&ctx->csr_buf, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, FRNN_ERR_OUT_OF_MEMORY, "cudaMalloc of the compact-output staging failed");
        }
        ctx->csr_bytes = need;
        ctx->held += need;
    }
    char* b = static_cast<char*>(ctx->csr_buf);
    ctx->csr_cnt = reinterpret_cast<int32_t*>(b);
    ctx->csr_idx = reinterpret_cast<int32_t*>(b + b_cnt);
    ctx->csr_d2 = reinterpret_cast<float*>(b + b_cnt + b_stage);
    ctx->csr_parts = reinterpret_cast<int64_t*>(b + b_cnt + 2 * b_stage);
    return FRNN_OK;
}

// The count pass of the compact output, enqueued: the search with staged
// rows, the offset scan, and the copy of the edge count into page-locked
// *h_edges (valid once the stream reaches it).  q: the search's launch.
static frnn_status csr_count_enqueue(frnn_ctx* ctx, const frnn_grid* grid, const float* queries,
                                     int64_t M, float r, int K, unsigned flags, int64_t* offsets,
                                     int32_t* degree, int64_t** h_edges, QueryLaunch* q) {
    if (!grid || grid->ctx != ctx) return fail(ctx, FRNN_ERR_INVALID_ARG, "grid is not of ctx");
    int32_t dummy = 0;   // check_query_args wants row outputs: the staging is ours
    frnn_status s = check_query_args(ctx, M, r, K, flags, &dummy, &dummy, reinterpret_cast<float*>(&dummy));
    if (s != FRNN_OK) return s;
    s = csr_reserve(ctx, M);
    if (s != FRNN_OK) return s;
    *q = QueryLaunch{};
    if (M > 0) {
        const CsrPass cp{degree};
        s = query_impl(ctx, grid, queries, M, r, K, flags, ctx->csr_cnt, ctx->csr_idx,
                       ctx->csr_d2, &cp, q);
        if (s != FRNN_OK) return s;
    }
    enqueue_csr_offsets(ctx->csr_cnt, M, ctx->csr_parts, offsets, ctx->stream);
    *h_edges = reinterpret_cast<int64_t*>(ctx->h_status + 2);
    cudaError_t e = cudaMemcpyAsync(*h_edges, offsets + M, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the edge count");
    return FRNN_OK;
}

frnn_status frnn_query_csr_count(frnn_ctx* ctx, const frnn_grid* grid, const float* queries,
                                 int64_t M, float r, int K, unsigned flags, int64_t* offsets,
                                 int32_t* degree, int64_t* n_edges) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    ctx->csr_pending = false;
    if (!offsets || !n_edges) return fail(ctx, FRNN_ERR_INVALID_ARG, "offsets or n_edges is NULL");
    *n_edges = 0;
    int64_t* h_edges = nullptr;
    QueryLaunch q{};
    frnn_status s = csr_count_enqueue(ctx, grid, queries, M, r, K, flags, offsets, degree, &h_edges, &q);
    if (s != FRNN_OK) return s;
    s = frnn_sync(ctx);
    if (s != FRNN_OK) return s;
    *n_edges = *h_edges;
    ctx->csr_q = q;
    ctx->csr_M = M;
    ctx->csr_E = *h_edges;
    ctx->csr_off = offsets;
    ctx->csr_pending = true;
    return FRNN_OK;
}

frnn_status frnn_query_csr_fill(frnn_ctx* ctx, int32_t* idx, float* dist2) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    if (!ctx->csr_pending)
        return fail(ctx, FRNN_ERR_INVALID_ARG,
                    "no pending frnn_query_csr_count on this context (or another call came between)");
    if (ctx->csr_E > 0 && (!idx || !dist2))
        return fail(ctx, FRNN_ERR_INVALID_ARG, "idx or dist2 is NULL");
    ctx->csr_pending = false;
    if (ctx->csr_M == 0) return FRNN_OK;
    enqueue_csr_gather(ctx->csr_cnt, ctx->csr_off, ctx->csr_idx, ctx->csr_d2, ctx->csr_M, idx,
                       dist2, ctx->num_sms, ctx->stream);
    QueryLaunch q = ctx->csr_q;
    q.ovf_mode = 2;
    q.row_off = ctx->csr_off;
    q.idx = idx;
    q.dist2 = dist2;
    q.degree = nullptr;
    std::string err;
    frnn_status s = enqueue_overflow_only(q, ctx->stream, err);
    if (s != FRNN_OK) return fail(ctx, s, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "compact-output gather launch");
    return FRNN_OK;
}

static bool same_events(const frnn_ctx* c, const frnn_event* ev, int n) {
    if ((int)c->g_ev.size() != n) return false;
    for (int e = 0; e < n; ++e) {
        const frnn_event& a = c->g_ev[e];
        const frnn_event& b = ev[e];
        if (a.pts != b.pts || a.n != b.n || a.counts != b.counts || a.idx != b.idx ||
            a.dist2 != b.dist2)
            return false;
    }
    return true;
}

// Path of one event of a batch: 0 grid scan by chunks, 2 grid scan by row
// tasks, 1 tensor core (autotuned per size class, else the defaults).
static int batch_path(const frnn_ctx* ctx, int64_t n, int D, int K, unsigned flags) {
    if (use_tc_path(ctx, D, flags, n, K)) return 1;
    return grid_kernel(build_naxes(ctx, n, D)) == 1 ? 2 : 0;
}

// ev: ordered by path (chunks, row tasks, tensor core), so that each path's
// events occupy one range of chunks, cell-array entries and slots.
static frnn_status enqueue_batched(frnn_ctx* ctx, const frnn_event* ev, int n_events, int D,
                                   float r, int K, unsigned flags, bool capturing,
                                   cudaStream_t st) {
    std::vector<const float*> refs(n_events);
    bool any_path[3] = {false, false, false};
    int first_rows = n_events, first_tc = n_events;   // first event of each later path
    for (int e = 0; e < n_events; ++e) {
        refs[e] = ev[e].pts;
        EventHdr& h = ctx->batch.h_hdr[e];
        h.counts = ev[e].counts;
        h.idx = ev[e].idx;
        h.dist2 = ev[e].dist2;
        // per event: autotuned cell multiple, axes and path for its size class
        h.m = build_mult(ctx, ev[e].n, D);
        h.naxes = build_naxes(ctx, ev[e].n, D);
        h.path = batch_path(ctx, ev[e].n, D, K, flags);
        if (ev[e].n > 0) any_path[h.path] = true;
        if (h.path != 0 && first_rows == n_events) first_rows = e;
        if (h.path == 1 && first_tc == n_events) first_tc = e;
    }
    const GridBufs& gb = ctx->batch;
    const auto slot_of = [&](int e) { return e < n_events ? gb.h_hdr[e].pt_off : gb.n_total; };
    const bool any_grid = any_path[0], any_rows = any_path[2], any_tc = any_path[1];
    BuildOpts o;
    o.r = r;
    o.m = 1;
    o.axes_mode = ctx->axes_mode;
    std::string err;
    frnn_status s = enqueue_build(ctx->batch, refs.data(), o, nullptr, ctx->d_status, st,
                                  capturing, err);
    if (s != FRNN_OK) return fail(ctx, s, err);
    QueryLaunch q{};
    q.qset = &ctx->batch;
    q.rset = &ctx->batch;
    q.r2 = r * r;
    q.K = K;
    q.self = 1;
    q.exit_dims = ctx->exit_dims;
    q.stage = ctx->staging == 2 ? 1 : 0;
    q.d_status = ctx->d_status;
    q.num_sms = ctx->num_sms;
    const bool mixed = (int)any_grid + (int)any_rows + (int)any_tc > 1;
    if (any_grid || (!any_tc && !any_rows)) {
        q.kernel = 0;
        q.path_filter = mixed ? 0 : -1;
        // the chunks of the chunk-scan events only
        if (mixed && first_rows < n_events) q.chunk_end = gb.h_hdr[first_rows].qchunk0;
        s = enqueue_grid_query(q, st, err);
        if (s != FRNN_OK) return fail(ctx, s, err);
    }
    if (any_rows) {
        // buffers were reserved before any capture; enqueue their build
        s = mixed ? rows_prepare(ctx->batch, ctx->d_status, st, err, 2, gb.h_cell_off[first_rows],
                                 gb.h_cell_off[first_tc], slot_of(first_rows), slot_of(first_tc))
                  : rows_prepare(ctx->batch, ctx->d_status, st, err);
        if (s != FRNN_OK) return fail(ctx, s, err);
        q.kernel = 1;
        q.chunk_end = -1;
        q.path_filter = mixed ? 2 : -1;
        s = enqueue_grid_query(q, st, err);
        if (s != FRNN_OK) return fail(ctx, s, err);
        q.kernel = 0;
    }
    if (any_tc) {
        // operands were allocated before any capture; enqueue their build
        s = mixed ? tc_prepare(ctx->batch, ctx->batch, ctx->d_status, st, err, 1,
                               gb.h_cell_off[first_tc], gb.h_cell_off[n_events])
                  : tc_prepare(ctx->batch, ctx->batch, ctx->d_status, st, err);
        if (s != FRNN_OK) return fail(ctx, s, err);
        q.tc_stats = ctx->d_tcstat;
        q.path_filter = mixed ? 1 : -1;
        s = enqueue_tc_query(q, st, err);
    }
    if (s != FRNN_OK) return fail(ctx, s, err);
    return FRNN_OK;
}

// Replay the captured graph on the internal stream, ordered after the work
// already on the context's stream and before anything enqueued there later.
static frnn_status launch_graph(frnn_ctx* ctx) {
    cudaError_t e = cudaEventRecord(ctx->g_in, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->gstream, ctx->g_in, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ctx->graph, ctx->gstream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->g_out, ctx->gstream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->g_out, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    return FRNN_OK;
}

frnn_status frnn_query_batched(frnn_ctx* ctx, const frnn_event* ev, int n_events, int D,
                               float r, int K, unsigned flags) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    ctx->csr_pending = false;
    if (n_events < 0 || (n_events > 0 && !ev))
        return fail(ctx, FRNN_ERR_INVALID_ARG, "bad event list");
    if (D < 1 || D > kMaxD) return fail(ctx, FRNN_ERR_INVALID_ARG, "D must be in 1..16");
    if (K < 1 || K > kMaxK) return fail(ctx, FRNN_ERR_INVALID_ARG, "K must be in 1..1024");
    if (!radius_ok(r)) return fail(ctx, FRNN_ERR_INVALID_ARG, "r must be finite, 2^-60..2^60");
    if (flags & ~(FRNN_SELF_QUERY | FRNN_PATH_GRID | FRNN_PATH_TC))
        return fail(ctx, FRNN_ERR_INVALID_ARG, "unknown flag bits");
    if ((flags & FRNN_PATH_TC) && D < 8)
        return fail(ctx, FRNN_ERR_UNSUPPORTED, "the tensor-core path needs D >= 8");
    if (n_events == 0) return FRNN_OK;
    for (int e = 0; e < n_events; ++e) {
        const frnn_event& x = ev[e];
        if (x.n < 0 || x.n >= INT32_MAX) return fail(ctx, FRNN_ERR_INVALID_ARG, "event n");
        if (x.n > 0 && (!x.pts || !x.counts || !x.idx || !x.dist2))
            return fail(ctx, FRNN_ERR_INVALID_ARG, "event pointer is NULL");
    }
    const frnn_event* caller_ev = ev;
    const int opts[5] = {ctx->cell_mult, ctx->axes_mode, ctx->exit_dims, ctx->grid_naxes,
                         ctx->staging};
    const bool hit = ctx->use_graph && ctx->graph && same_events(ctx, ev, n_events) &&
                     ctx->g_D == D && ctx->g_K == K && ctx->g_r == r && ctx->g_flags == flags &&
                     std::memcmp(opts, ctx->g_opts, sizeof(opts)) == 0;
    if (hit) return launch_graph(ctx);
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
        ctx->g_ev.clear();
    }
    // the batch in path order (chunk scan, row-task scan, tensor core; stable
    // within a path): each path's preparation and launch then covers only
    // its own events' chunks, cells and slots
    std::vector<frnn_event> ordered;
    ordered.reserve(n_events);
    for (int want : {0, 2, 1})
        for (int e = 0; e < n_events; ++e)
            if (batch_path(ctx, ev[e].n, D, K, flags) == want) ordered.push_back(ev[e]);
    ev = ordered.data();
    std::vector<int64_t> n(n_events);
    for (int e = 0; e < n_events; ++e) n[e] = ev[e].n;
    frnn_status s = alloc_accounted(ctx, ctx->batch, n_events, n.data(), D, nullptr);
    if (s != FRNN_OK) return s;
    bool batch_tc = false, batch_rows = false;
    for (int e = 0; e < n_events; ++e) {
        if (ev[e].n <= 0) continue;
        if (use_tc_path(ctx, D, flags, ev[e].n, K)) batch_tc = true;
        else if (grid_kernel(build_naxes(ctx, ev[e].n, D)) == 1) batch_rows = true;
    }
    if (batch_tc) {
        // allocate the tensor-core operands outside any capture (no work enqueued)
        std::string err;
        s = tc_reserve(ctx->batch, err);
        if (s != FRNN_OK) return fail(ctx, s, err);
    }
    if (batch_rows) {
        // the row-task kernel's buffers likewise
        const size_t before = ctx->batch.rows_bytes;
        std::string err;
        s = rows_reserve(ctx->batch, err);
        ctx->held = ctx->held - std::min(ctx->held, before) + ctx->batch.rows_bytes;
        if (s != FRNN_OK) return fail(ctx, s, err);
    }
    if (!ctx->use_graph)
        return enqueue_batched(ctx, ev, n_events, D, r, K, flags, false, ctx->stream);
    if (!ctx->gstream) {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->g_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->g_out, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph stream setup");
    }
    // the pinned table mirror must be free before its upload is captured, and
    // the previous replay must be done before the tables change
    cudaStreamSynchronize(ctx->gstream);
    if (ctx->batch.h_pinned_free) cudaEventSynchronize(ctx->batch.h_pinned_free);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    s = enqueue_batched(ctx, ev, n_events, D, r, K, flags, true, ctx->gstream);
    e = cudaStreamEndCapture(ctx->gstream, &graph);
    if (s != FRNN_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    ctx->graph = exec;
    ctx->g_ev.assign(caller_ev, caller_ev + n_events);
    ctx->g_D = D;
    ctx->g_K = K;
    ctx->g_r = r;
    ctx->g_flags = flags;
    std::memcpy(ctx->g_opts, opts, sizeof(opts));
    return launch_graph(ctx);
}

frnn_status frnn_self_query_host(frnn_ctx* ctx, const float* refs_host, int64_t N, int D,
                                 float r, int K, unsigned flags, int32_t* counts_host,
                                 int32_t* idx_host, float* dist2_host) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    if (D < 1 || D > kMaxD) return fail(ctx, FRNN_ERR_INVALID_ARG, "D must be in 1..16");
    frnn_status s = check_query_args(ctx, N, r, K, flags | FRNN_SELF_QUERY, counts_host,
                                     idx_host, dist2_host);
    if (s != FRNN_OK) return s;
    if (N > 0 && !refs_host) return fail(ctx, FRNN_ERR_INVALID_ARG, "refs_host is NULL");
    if (N == 0) return FRNN_OK;
    const size_t b_in = sizeof(float) * (size_t)N * D;
    const size_t b_cnt = sizeof(int32_t) * (size_t)N;
    const size_t b_row = sizeof(int32_t) * (size_t)N * K;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    // page-locked outputs: the query writes them directly (no staging, no
    // copy; 1.07 vs 1.31 ms end to end for the 300k x 8 event, K = 64)
    int32_t* m_cnt = static_cast<int32_t*>(mapped_host(counts_host));
    int32_t* m_idx = static_cast<int32_t*>(mapped_host(idx_host));
    float* m_d2 = static_cast<float*>(mapped_host(dist2_host));
    const bool direct = m_cnt && m_idx && m_d2;
    const size_t need = al(b_in) + (direct ? 0 : al(b_cnt) + 2 * al(b_row));
    if (need > ctx->hp_bytes) {
        if (!budget_allows(ctx, ctx->hp_bytes, need))
            return fail(ctx, FRNN_ERR_BUDGET, "request exceeds the context's memory budget");
        cudaStreamSynchronize(ctx->stream);
        if (ctx->hp_buf) cudaFree(ctx->hp_buf);
        ctx->held -= std::min(ctx->held, ctx->hp_bytes);
        ctx->hp_buf = nullptr;
        ctx->hp_bytes = 0;
        if (cudaMalloc(&ctx->hp_buf, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, FRNN_ERR_OUT_OF_MEMORY, "cudaMalloc of host-path buffers failed");
        }
        ctx->hp_bytes = need;
        ctx->held += need;
    }
    char* b = static_cast<char*>(ctx->hp_buf);
    float* d_in = reinterpret_cast<float*>(b);
    int32_t* d_cnt = direct ? m_cnt : reinterpret_cast<int32_t*>(b + al(b_in));
    int32_t* d_idx = direct ? m_idx : reinterpret_cast<int32_t*>(b + al(b_in) + al(b_cnt));
    float* d_d2 = direct ? m_d2
                         : reinterpret_cast<float*>(b + al(b_in) + al(b_cnt) + al(b_row));
    cudaError_t e = cudaMemcpyAsync(d_in, refs_host, b_in, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "H2D copy");
    release_host_grid_if_other_dim(ctx, D);
    s = frnn_build_grid(ctx, d_in, N, D, r, &ctx->host_grid);
    if (s != FRNN_OK) return s;
    s = frnn_query(ctx, ctx->host_grid, d_in, N, r, K, flags | FRNN_SELF_QUERY, d_cnt, d_idx,
                   d_d2);
    if (s != FRNN_OK) return s;
    if (direct) return frnn_sync(ctx);
    cudaMemcpyAsync(counts_host, d_cnt, b_cnt, cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(idx_host, d_idx, b_row, cudaMemcpyDeviceToHost, ctx->stream);
    e = cudaMemcpyAsync(dist2_host, d_d2, b_row, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "D2H copy");
    return frnn_sync(ctx);
}

// Grow one of the context's device buffers of the host-buffer path (charged
// to the budget; the stream is drained before the old buffer is freed).
static frnn_status grow(frnn_ctx* ctx, void*& buf, size_t& bytes, size_t need, const char* what) {
    if (need <= bytes) return FRNN_OK;
    if (!budget_allows(ctx, bytes, need))
        return fail(ctx, FRNN_ERR_BUDGET, "request exceeds the context's memory budget");
    cudaStreamSynchronize(ctx->stream);
    if (buf) cudaFree(buf);
    ctx->held -= std::min(ctx->held, bytes);
    buf = nullptr;
    bytes = 0;
    if (cudaMalloc(&buf, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FRNN_ERR_OUT_OF_MEMORY, std::string("cudaMalloc of ") + what + " failed");
    }
    bytes = need;
    ctx->held += need;
    return FRNN_OK;
}

frnn_status frnn_self_query_host_csr(frnn_ctx* ctx, const float* refs_host, int64_t N, int D,
                                     float r, int K, unsigned flags, int64_t* offsets_host,
                                     int32_t* idx_host, float* dist2_host, int64_t edge_cap,
                                     int64_t* n_edges) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    if (D < 1 || D > kMaxD) return fail(ctx, FRNN_ERR_INVALID_ARG, "D must be in 1..16");
    if (!offsets_host || !n_edges || edge_cap < 0)
        return fail(ctx, FRNN_ERR_INVALID_ARG, "offsets_host or n_edges is NULL, or edge_cap < 0");
    if (edge_cap > 0 && (!idx_host || !dist2_host))
        return fail(ctx, FRNN_ERR_INVALID_ARG, "idx_host or dist2_host is NULL");
    int32_t dummy = 0;
    frnn_status s = check_query_args(ctx, N, r, K, flags | FRNN_SELF_QUERY, &dummy, &dummy,
                                     reinterpret_cast<float*>(&dummy));
    if (s != FRNN_OK) return s;
    if (N > 0 && !refs_host) return fail(ctx, FRNN_ERR_INVALID_ARG, "refs_host is NULL");
    *n_edges = 0;
    if (N == 0) {
        offsets_host[0] = 0;
        return FRNN_OK;
    }
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t b_in = sizeof(float) * (size_t)N * D;
    const size_t b_off = sizeof(int64_t) * (size_t)(N + 1);
    s = grow(ctx, ctx->hp_buf, ctx->hp_bytes, al(b_in) + al(b_off), "host-path buffers");
    if (s != FRNN_OK) return s;
    float* d_in = static_cast<float*>(ctx->hp_buf);
    int64_t* d_off = reinterpret_cast<int64_t*>(static_cast<char*>(ctx->hp_buf) + al(b_in));
    cudaError_t e = cudaMemcpyAsync(d_in, refs_host, b_in, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "H2D copy");
    release_host_grid_if_other_dim(ctx, D);
    s = frnn_build_grid(ctx, d_in, N, D, r, &ctx->host_grid);
    if (s != FRNN_OK) return s;
    // The count pass, then the fill before the host has read the edge count
    // back: the device rows are sized for the caller's capacity (at most N K
    // entries), and nothing is written past it (the call fails when the count
    // exceeds it).  The fill runs in kParts ranges of rows, each copied back
    // on a copy stream while the next range is gathered; the offsets go back
    // as soon as the scan has made them.  Beyond kEarlyGatherBytes of rows,
    // or beyond the context's memory budget, the fill waits for the count,
    // is sized by it and is copied back after it.
    constexpr int kParts = 4;
    ctx->csr_pending = false;
    int64_t* h_edges = nullptr;
    QueryLaunch q{};
    s = csr_count_enqueue(ctx, ctx->host_grid, d_in, N, r, K, flags | FRNN_SELF_QUERY, d_off,
                          nullptr, &h_edges, &q);
    if (s != FRNN_OK) return s;
    // the offsets at the parts' first rows (multiples of 32), to the pinned
    // block's next slots
    int64_t cut[kParts + 1];
    cut[0] = 0;
    cut[kParts] = N;
    for (int p = 1; p < kParts; ++p) cut[p] = std::min<int64_t>(N, (N * p / kParts + 31) / 32 * 32);
    int64_t* h_cut = h_edges + 1;
    for (int p = 1; p < kParts && e == cudaSuccess; ++p)
        e = cudaMemcpyAsync(h_cut + (p - 1), d_off + cut[p], sizeof(int64_t), cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the part offsets");
    if (!ctx->ev_edges) {
        e = cudaEventCreateWithFlags(&ctx->ev_edges, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "event for the edge count");
    }
    e = cudaEventRecord(ctx->ev_edges, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event for the edge count");
    constexpr size_t kEarlyGatherBytes = size_t(1) << 30;
    const int64_t cap = std::min<int64_t>(edge_cap, N * (int64_t)K);
    const size_t early_bytes = 2 * al(sizeof(int32_t) * (size_t)std::max<int64_t>(cap, 1));
    // (within the context's memory budget too: else the rows wait for the
    // count, which may need fewer bytes)
    const bool early = early_bytes <= kEarlyGatherBytes &&
                       (early_bytes <= ctx->hr_bytes || budget_allows(ctx, ctx->hr_bytes, early_bytes));
    int32_t* d_idx = nullptr;
    float* d_d2 = nullptr;
    auto rows_buffers = [&](int64_t entries) -> frnn_status {
        const size_t b_rows = al(sizeof(int32_t) * (size_t)std::max<int64_t>(entries, 1));
        // the rows are gathered in HBM and copied back by the copy engine
        // (measured faster here than gathering straight into page-locked
        // host memory: 0.82 vs 0.95 ms for the 300k x 8 event)
        frnn_status st = grow(ctx, ctx->hr_buf, ctx->hr_bytes, 2 * b_rows, "compact host-path rows");
        if (st != FRNN_OK) return st;
        d_idx = static_cast<int32_t*>(ctx->hr_buf);
        d_d2 = reinterpret_cast<float*>(static_cast<char*>(ctx->hr_buf) + b_rows);
        return FRNN_OK;
    };
    // the selection kernel's rows (longer than the in-kernel list), then the
    // gather of the others
    auto fill = [&](int64_t rows_cap, bool in_parts) -> frnn_status {
        QueryLaunch qf = q;
        qf.ovf_mode = 2;
        qf.row_off = d_off;
        qf.idx = d_idx;
        qf.dist2 = d_d2;
        qf.degree = nullptr;
        qf.row_cap = rows_cap;
        std::string err;
        frnn_status st = enqueue_overflow_only(qf, ctx->stream, err);
        if (st != FRNN_OK) return fail(ctx, st, err);
        for (int p = 0; p < (in_parts ? kParts : 1); ++p) {
            const int64_t r0 = in_parts ? cut[p] : 0, r1 = in_parts ? cut[p + 1] : N;
            enqueue_csr_gather(ctx->csr_cnt, d_off, ctx->csr_idx, ctx->csr_d2, N, d_idx, d_d2,
                               ctx->num_sms, ctx->stream, rows_cap, r0, r1);
            if (in_parts) cudaEventRecord(ctx->ev_part[p], ctx->stream);
        }
        const cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "compact-output fill launch");
        return FRNN_OK;
    };
    if (early) {
        if (!ctx->cstream) {
            e = cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking);
            for (cudaEvent_t& ev : ctx->ev_part)
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream of the compact host path");
        }
        s = rows_buffers(cap);
        if (s != FRNN_OK) return s;
        // the offsets go back while the rows are filled
        e = cudaStreamWaitEvent(ctx->cstream, ctx->ev_edges, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(offsets_host, d_off, b_off, cudaMemcpyDeviceToHost, ctx->cstream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "D2H copy");
        s = fill(cap, true);
        if (s != FRNN_OK) return s;
    }
    e = cudaEventSynchronize(ctx->ev_edges);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "waiting for the edge count");
    const int64_t E = *h_edges;
    *n_edges = E;
    if (E > edge_cap) {
        if (early) e = cudaStreamSynchronize(ctx->cstream);   // the offsets are on their way
        else e = cudaMemcpyAsync(offsets_host, d_off, b_off, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "D2H copy");
        s = frnn_sync(ctx);   // a device-side error takes precedence
        if (s != FRNN_OK) return s;
        return fail(ctx, FRNN_ERR_CAPACITY, "more edges than edge_cap (n_edges has the count)");
    }
    if (early) {
        // each part's entries, [offset of its first row, offset of the next
        // part's first row), once its gather is done
        for (int p = 0; p < kParts && e == cudaSuccess; ++p) {
            const int64_t a0 = p == 0 ? 0 : h_cut[p - 1];
            const int64_t a1 = p + 1 < kParts ? h_cut[p] : E;
            e = cudaStreamWaitEvent(ctx->cstream, ctx->ev_part[p], 0);
            if (e == cudaSuccess && a1 > a0)
                e = cudaMemcpyAsync(idx_host + a0, d_idx + a0, sizeof(int32_t) * (size_t)(a1 - a0),
                                    cudaMemcpyDeviceToHost, ctx->cstream);
            if (e == cudaSuccess && a1 > a0)
                e = cudaMemcpyAsync(dist2_host + a0, d_d2 + a0, sizeof(float) * (size_t)(a1 - a0),
                                    cudaMemcpyDeviceToHost, ctx->cstream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_copied, ctx->cstream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_copied, 0);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "D2H copy");
        return frnn_sync(ctx);
    }
    s = rows_buffers(E);
    if (s != FRNN_OK) return s;
    s = fill(E, false);
    if (s != FRNN_OK) return s;
    e = cudaMemcpyAsync(offsets_host, d_off, b_off, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && E > 0)
        e = cudaMemcpyAsync(idx_host, d_idx, sizeof(int32_t) * (size_t)E, cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e == cudaSuccess && E > 0)
        e = cudaMemcpyAsync(dist2_host, d_d2, sizeof(float) * (size_t)E, cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "D2H copy");
    return frnn_sync(ctx);
}

frnn_status frnn_check_wait_timeout(frnn_ctx* ctx, uint64_t limit_ns) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    if (limit_ns < 1000000ull || limit_ns > 5000000000ull)
        return fail(ctx, FRNN_ERR_INVALID_ARG, "limit_ns must be in [1e6, 5e9]");
    ctx->csr_pending = false;
    const cudaError_t e = launch_wait_timeout(limit_ns, ctx->d_status, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait-timeout check launch");
    return frnn_sync(ctx);
}

frnn_status frnn_sync(frnn_ctx* ctx) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
    const int32_t st = *ctx->h_status;
    if (st == 0) return FRNN_OK;
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (st & kStatusNonFinite)
        return fail(ctx, FRNN_ERR_NONFINITE, "an input coordinate is NaN or infinite");
    if (st & kStatusCapacity)
        return fail(ctx, FRNN_ERR_CAPACITY, "an internal device-side capacity overflowed");
    if (st & kStatusTimeout)
        return fail(ctx, FRNN_ERR_TIMEOUT, "a bounded device-side wait ran out");
    return fail(ctx, FRNN_ERR_CUDA, "unknown device status");
}

const char* frnn_last_error(const frnn_ctx* ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

frnn_status frnn_autotune(frnn_ctx* ctx, const float* refs, int64_t N, int D, float r, int K,
                          unsigned flags, frnn_tune_result* best) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    if (D < 1 || D > kMaxD) return fail(ctx, FRNN_ERR_INVALID_ARG, "D must be in 1..16");
    if (N < 1 || N >= INT32_MAX || !refs)
        return fail(ctx, FRNN_ERR_INVALID_ARG, "autotune needs N >= 1 device points");
    if (K < 1 || K > kMaxK) return fail(ctx, FRNN_ERR_INVALID_ARG, "K must be in 1..1024");
    if (!radius_ok(r)) return fail(ctx, FRNN_ERR_INVALID_ARG, "r must be finite, 2^-60..2^60");
    const size_t ob = (size_t)N * (sizeof(int32_t) + (size_t)K * 8);
    if (!budget_allows(ctx, 0, ob)) return fail(ctx, FRNN_ERR_BUDGET, "autotune outputs exceed budget");
    void* out = nullptr;
    if (cudaMalloc(&out, ob) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FRNN_ERR_OUT_OF_MEMORY, "autotune outputs");
    }
    int32_t* counts = static_cast<int32_t*>(out);
    int32_t* idx = counts + N;
    float* dist2 = reinterpret_cast<float*>(idx + (size_t)N * K);
    // each timed run starts with the L2 cache flushed (a write larger than it,
    // not timed), as a run over many events or after other work would
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device);
    const size_t flush_bytes = std::max<size_t>(2 * (size_t)std::max(l2, 0), 1 << 20);
    void* flush = nullptr;
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        flush = nullptr;   // timed without the flush
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_m = ctx->cell_mult, saved_x = ctx->exit_dims, saved_a = ctx->grid_naxes,
              saved_s = ctx->staging;
    frnn_tune_result bestr{FRNN_PATH_GRID, 1, 0, INFINITY, 0, 1};
    frnn_status s = FRNN_OK;
    frnn_grid* g = nullptr;
    auto timed = [&](auto&& fn, float& ms) -> frnn_status {
        float bestms = INFINITY;
        for (int rep = 0; rep < 4; ++rep) {   // first run warms up
            if (flush) cudaMemsetAsync(flush, rep, flush_bytes, ctx->stream);
            cudaEventRecord(e0, ctx->stream);
            frnn_status st = fn();
            if (st != FRNN_OK) return st;
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) return FRNN_ERR_CUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) bestms = std::min(bestms, t);
        }
        ms = bestms;
        return frnn_sync(ctx);
    };
    // grid configurations: the automatic axis choice (five axes, or four
    // when the cell budget makes five-axis cells too coarse; chunk kernel),
    // four axes with cells of r and three with cells of r/2 (row-task
    // kernel); fewer for smaller D.  Cells of r/2 and r/3 on the automatic
    // choice too, where its (2m + 1)^(axes - 1) neighbour rows stay within
    // the chunk kernel's table (m = 2 up to D = 4, m = 3 up to D = 3):
    // beyond that the grid lowers m and the configuration repeats another
    struct GridCfg { int naxes, m; };
    std::vector<GridCfg> gcfg;
    auto add_cfg = [&](int na, int m) {
        if (na > 0) na = std::min(na, D);
        for (const GridCfg& c : gcfg)
            if (c.naxes == na && c.m == m) return;
        gcfg.push_back({na, m});
    };
    add_cfg(0, 1);
    add_cfg(4, 1);
    add_cfg(3, 2);
    for (int m = 2; m <= 3; ++m) {
        int rows = 1;
        for (int a = 1; a < std::min(D, kMaxAxes); ++a) rows *= 2 * m + 1;
        if (rows <= kMaxNbrRows) add_cfg(0, m);
    }
    for (size_t gi = 0; gi < gcfg.size() && s == FRNN_OK; ++gi) {
        const int m = gcfg[gi].m;
        ctx->cell_mult = m;
        ctx->grid_naxes = gcfg[gi].naxes;
        // the chunk kernel with either staging; the row-task kernel with its
        // default vote point and a later one
        struct Cand { unsigned path; int staging, exit_dims; };
        std::vector<Cand> cands;
        if (!(flags & FRNN_PATH_TC)) {
            if (grid_kernel(gcfg[gi].naxes) == 0) {
                cands.push_back({FRNN_PATH_GRID, 1, 0});
                cands.push_back({FRNN_PATH_GRID, 2, 0});
            } else {
                cands.push_back({FRNN_PATH_GRID, 1, 0});
                if (D >= 5) cands.push_back({FRNN_PATH_GRID, 1, 3});
            }
        }
        if (D >= 8 && !(flags & FRNN_PATH_GRID)) cands.push_back({FRNN_PATH_TC, 1, 0});
        if (cands.empty()) {
            s = fail(ctx, FRNN_ERR_UNSUPPORTED, "the tensor-core path needs D >= 8");
            break;
        }
        // each run is a whole step, build then query: a query's per-build
        // preparation (the row-task scan's pair copy and task list, the
        // tensor-core operands) is timed with it
        for (const Cand& c : cands) {
            ctx->staging = c.staging;
            ctx->exit_dims = c.exit_dims;
            float ms = 0.f;
            s = timed([&] {
                frnn_status st = frnn_build_grid(ctx, refs, N, D, r, &g);
                if (st != FRNN_OK) return st;
                return frnn_query(ctx, g, refs, N, r, K, FRNN_SELF_QUERY | c.path, counts, idx,
                                  dist2);
            }, ms);
            if (s != FRNN_OK) break;
            if (ms < bestr.ms) bestr = {(int)c.path, m, c.exit_dims, ms, gcfg[gi].naxes, c.staging};
        }
    }
    ctx->cell_mult = saved_m;
    ctx->exit_dims = saved_x;
    ctx->grid_naxes = saved_a;
    ctx->staging = saved_s;
    if (g) frnn_grid_destroy(g);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (flush) cudaFree(flush);
    if (s != FRNN_OK) return s;
    ctx->tuned[tune_key(N, D, K)] = {bestr.path == FRNN_PATH_TC ? 1 : 0, bestr.cell_mult,
                                     bestr.exit_dims, bestr.ms, bestr.grid_axes, bestr.staging};
    if (ctx->graph) {   // captured batches may now take other paths
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
        ctx->g_ev.clear();
    }
    if (best) *best = bestr;
    return FRNN_OK;
}

frnn_status frnn_set_option(frnn_ctx* ctx, frnn_option opt, int64_t value) {
    if (!ctx) return FRNN_ERR_INVALID_ARG;
    switch (opt) {
        case FRNN_OPT_CELL_MULT:
            if (value < 0 || value > 3)
                return fail(ctx, FRNN_ERR_INVALID_ARG, "m must be 0 (tuned), 1, 2 or 3");
            ctx->cell_mult = (int)value;
            return FRNN_OK;
        case FRNN_OPT_GRID_AXES:
            if (value < 0 || value > 1) return fail(ctx, FRNN_ERR_INVALID_ARG, "axes mode 0 or 1");
            ctx->axes_mode = (int)value;
            return FRNN_OK;
        case FRNN_OPT_GRID_NAXES:
            if (value < 0 || value > kMaxAxes)
                return fail(ctx, FRNN_ERR_INVALID_ARG, "gridded axes must be 0 (tuned) or 1..5");
            ctx->grid_naxes = (int)value;
            return FRNN_OK;
        case FRNN_OPT_EXIT_DIMS:
            if (value < 0 || value > kMaxD) return fail(ctx, FRNN_ERR_INVALID_ARG, "exit dims");
            ctx->exit_dims = (int)value;
            return FRNN_OK;
        case FRNN_OPT_STAGING:
            if (value < 0 || value > 2)
                return fail(ctx, FRNN_ERR_INVALID_ARG, "staging must be 0 (tuned), 1 or 2");
            ctx->staging = (int)value;
            return FRNN_OK;
        case FRNN_OPT_USE_GRAPH:
            ctx->use_graph = value ? 1 : 0;
            return FRNN_OK;
        case FRNN_OPT_AUTOTUNE:
            // 0 also forgets every tuned configuration
            ctx->autotune = value ? 1 : 0;
            if (!value) ctx->tuned.clear();
            return FRNN_OK;
        case FRNN_OPT_AUTO_TC:
            ctx->auto_tc = value ? 1 : 0;
            return FRNN_OK;
        case FRNN_OPT_TC_SURVIVORS:
        case FRNN_OPT_TC_ACCEPTED:
            cudaStreamSynchronize(ctx->stream);
            cudaMemset(ctx->d_tcstat, 0, 2 * sizeof(unsigned long long));
            return FRNN_OK;
        case FRNN_OPT_KERNEL_TIMING:
            cudaStreamSynchronize(ctx->stream);
            ctx->ktime = value ? 1 : 0;
            ctx->kev_used = 0;
            return FRNN_OK;
    }
    return fail(ctx, FRNN_ERR_INVALID_ARG, "unknown option");
}

frnn_status frnn_kernel_times(frnn_ctx* ctx, float* ms, int max, int* n) {
    if (!ctx || !n || max < 0 || (max > 0 && !ms)) return FRNN_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
    const int used = ctx->kev_used;
    ctx->kev_used = 0;
    for (int i = 0; i < used && i < max; ++i) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ctx->kev[2 * i], ctx->kev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel timing event");
        ms[i] = t;
    }
    *n = used;
    return FRNN_OK;
}

frnn_status frnn_get_option(const frnn_ctx* ctx, frnn_option opt, int64_t* value) {
    if (!ctx || !value) return FRNN_ERR_INVALID_ARG;
    switch (opt) {
        case FRNN_OPT_CELL_MULT: *value = ctx->cell_mult; return FRNN_OK;
        case FRNN_OPT_GRID_AXES: *value = ctx->axes_mode; return FRNN_OK;
        case FRNN_OPT_GRID_NAXES: *value = ctx->grid_naxes; return FRNN_OK;
        case FRNN_OPT_EXIT_DIMS: *value = ctx->exit_dims; return FRNN_OK;
        case FRNN_OPT_STAGING: *value = ctx->staging; return FRNN_OK;
        case FRNN_OPT_USE_GRAPH: *value = ctx->use_graph; return FRNN_OK;
        case FRNN_OPT_AUTOTUNE: *value = ctx->autotune; return FRNN_OK;
        case FRNN_OPT_AUTO_TC: *value = ctx->auto_tc; return FRNN_OK;
        case FRNN_OPT_KERNEL_TIMING: *value = ctx->ktime; return FRNN_OK;
        case FRNN_OPT_TC_SURVIVORS:
        case FRNN_OPT_TC_ACCEPTED: {
            unsigned long long h[2] = {0, 0};
            cudaStreamSynchronize(ctx->stream);
            if (cudaMemcpy(h, ctx->d_tcstat, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
                return FRNN_ERR_CUDA;
            *value = (int64_t)(opt == FRNN_OPT_TC_SURVIVORS ? h[0] : h[1]);
            return FRNN_OK;
        }
    }
    return FRNN_ERR_INVALID_ARG;
}

}  // extern "C"
