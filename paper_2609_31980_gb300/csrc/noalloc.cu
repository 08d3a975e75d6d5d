// noalloc.cu — a self-query that allocates nothing.
//
// Some callers cannot allocate memory when they run a query: code that runs
// under a fixed, pre-reserved memory plan (an embedded or real-time host
// loop that must not call into the allocator, a process whose device memory
// is carved up in advance among several engines), or code between the
// launches of a latency-critical pipeline, where cudaMalloc or cudaFree
// would synchronise the whole device.  frnn_self_query_noalloc serves them:
// its grid and counters live in one fixed-size array in device memory that
// the library declares at file scope, so the call issues no cudaMalloc,
// cudaFree, page-locked allocation or library allocation at all; the caller
// provides the points and the output rows.  The call is synchronous: it
// waits for its own work and reads the device status word back.
//
// The array holds the grid of at most kNoAllocMaxPoints points in up to 16
// dimensions (about 7 MB).  Every GPU that loads the library keeps it until
// the process exits.  All calls share it and each call leaves its own
// contents there; the kernels clear what must start at zero.  Two calls whose
// work overlaps on the GPU (other streams, other host threads) race on the
// array and give wrong results: serialise them.
//
// In host code the array's name stands for a host-side shadow, not a device
// address; every call looks the device address up with cudaGetSymbolAddress,
// with the caller's device current, and passes that pointer to the kernels.
// The first call on a device also loads the library's device code there,
// which places the array; make that first call before any stream capture
// begins.  Looking the address up on every call (instead of caching it)
// keeps it right after a device reset, which places the array anew.
#include <string>

#include "frnn_host.h"

namespace frnn {

constexpr int64_t kNoAllocMaxPoints = 65536;

constexpr int64_t na_cap(int64_t n) {
    return (n / 2 + 1 > 16384 ? n / 2 + 1 : 16384) > ((int64_t)1 << 24)
               ? ((int64_t)1 << 24)
               : (n / 2 + 1 > 16384 ? n / 2 + 1 : 16384);
}
constexpr size_t na_al(size_t x) { return (x + 255) / 256 * 256; }
// bytes of the grid of one n-point event in D dimensions, carved as below
constexpr size_t na_bytes(int64_t n, int D) {
    const int64_t cn = ((n + 1) & ~(int64_t)1) > 0 ? ((n + 1) & ~(int64_t)1) : 1;
    const int64_t L = na_cap(n) + 1;
    const int64_t parts = (L + kScanChunk - 1) / kScanChunk > 0 ? (L + kScanChunk - 1) / kScanChunk : 1;
    return na_al(sizeof(EventHdr)) + na_al(sizeof(int32_t) * 2) + na_al(sizeof(int64_t) * 2) +
           na_al(sizeof(int32_t) * kBBoxStride * kBBoxCopies) +
           na_al(sizeof(float) * padded_dim(D) * (cn + kTcRowPad)) + 4 * na_al(sizeof(int32_t) * cn) +
           na_al(sizeof(int32_t) * L) + na_al(sizeof(Overflow) * cn) + na_al(sizeof(int32_t) * kScalars) +
           na_al(sizeof(int32_t) * parts) + na_al(sizeof(int32_t) * 16);   // + status word
}
constexpr size_t kNoAllocBytes = na_bytes(kNoAllocMaxPoints, kMaxD);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// the per-event tables the host would otherwise upload, and a clean status word
__global__ void k_noalloc_tables(EventHdr* hdr, int32_t* blk_start, int64_t* cell_off,
                                 const float* pts, int64_t n, int32_t cap, int32_t nblk,
                                 int32_t* status) {
    if (threadIdx.x != 0) return;
    EventHdr h{};
    h.refs = pts;
    h.n = n;
    h.pt_off = 0;
    h.cell_off = 0;
    h.cell_cap = cap;
    h.valid = 1;
    *hdr = h;
    blk_start[0] = 0;
    blk_start[1] = nblk;
    cell_off[0] = 0;
    cell_off[1] = cap + 1;
    *status = 0;
}

// Point the arrays of a one-event GridBufs into the scratch (same layout rules
// as the allocating path); returns the status word's address.
static int32_t* carve(GridBufs& g, char* b, int64_t n, int D) {
    const int64_t cn = std::max<int64_t>((n + 1) & ~(int64_t)1, 1);
    const int64_t cap = na_cap(n);
    g.E = 1;
    g.D = D;
    g.DP = padded_dim(D);
    g.n_total = (n + 1) & ~(int64_t)1;
    g.L = cap + 1;
    g.nblk = std::max<int64_t>(1, ceil_div(n, kBuildPtsPerBlock));
    g.nparts = scan_parts_needed(g.L);
    g.nchunks = ceil_div(n, kChunkQ);   // the header's first chunk is 0
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = b + off;
        off += na_al(bytes);
        return p;
    };
    g.hdr = reinterpret_cast<EventHdr*>(take(sizeof(EventHdr)));
    g.blk_start = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 2));
    g.cell_off = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * 2));
    g.bbox = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kBBoxStride * kBBoxCopies));
    g.pts = reinterpret_cast<float*>(take(sizeof(float) * g.DP * (cn + kTcRowPad)));
    g.perm = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cn));
    g.cell = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cn));
    g.cid = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cn));
    g.rnk = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cn));
    g.cstart = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * g.L));
    g.ovf = reinterpret_cast<Overflow*>(take(sizeof(Overflow) * cn));
    g.scalars = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kScalars));
    g.parts = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * g.nparts));
    return reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 16));
}

// Device address of the scratch array on the current device, or NULL.  The
// lookup allocates nothing once the device code is loaded.
static void* scratch_address() {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

}  // namespace frnn

using namespace frnn;

extern "C" {

frnn_status frnn_self_query_noalloc(const float* pts, int64_t N, int D, float r, int K,
                                    int32_t* counts, int32_t* idx, float* dist2,
                                    void* cuda_stream) {
    if (N < 0 || N > kNoAllocMaxPoints) return FRNN_ERR_INVALID_ARG;   // beyond the scratch
    if (D < 1 || D > kMaxD || K < 1 || K > kMaxK || !(r >= 0x1p-60f && r <= 0x1p60f))
        return FRNN_ERR_INVALID_ARG;
    if (N > 0 && (!pts || !counts || !idx || !dist2)) return FRNN_ERR_INVALID_ARG;
    if (N == 0) return FRNN_OK;
    std::string err;   // text of the build/launch helpers; only filled on an error path
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    char* base = static_cast<char*>(scratch_address());
    if (!base) return FRNN_ERR_CUDA;
    GridBufs g;
    int32_t* status = carve(g, base, N, D);
    k_noalloc_tables<<<1, 32, 0, st>>>(g.hdr, g.blk_start, g.cell_off, pts, N,
                                      (int32_t)na_cap(N), (int32_t)g.nblk, status);
    BuildOpts o;
    o.r = r;
    o.m = 1;
    o.axes_mode = 0;
    frnn_status s = enqueue_build_resident(g, o, status, st, err);
    if (s != FRNN_OK) return s;
    QueryLaunch q{};
    q.qset = &g;
    q.rset = &g;
    q.r2 = r * r;
    q.K = K;
    q.self = 1;
    q.exit_dims = 0;
    q.counts = counts;
    q.idx = idx;
    q.dist2 = dist2;
    q.d_status = status;
    q.num_sms = sms;
    s = enqueue_grid_query(q, st, err);
    if (s != FRNN_OK) return s;
    // synchronous: read the device status word back (no allocation)
    int32_t h = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&h, status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FRNN_ERR_CUDA;
    }
    if (h & kStatusNonFinite) return FRNN_ERR_NONFINITE;
    if (h & kStatusCapacity) return FRNN_ERR_CAPACITY;
    if (h & kStatusTimeout) return FRNN_ERR_TIMEOUT;
    return FRNN_OK;
}

}  // extern "C"
