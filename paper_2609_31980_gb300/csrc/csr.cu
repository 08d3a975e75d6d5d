// csr.cu — count-first compact output (CSR rows).
//
// The paper keeps only the edges that exist: the search first fixes how many
// neighbours every query keeps, the caller allocates exactly that many
// entries, and the rows are then written back to back (Sec. 4, "count-first
// exact allocation", which cut the temporary edge buffer of the real event
// from 4.35 GB to 148 MB; "compact output" among the retained ideas).
//
// Here the search runs once.  Its kernels write every row (sorted, at most 32
// entries) into a staging area of the context, 32 entries per original query
// index, and its count into cnt[i]; rows longer than the in-kernel list are
// marked (kCsrSpill) and counted exactly by the selection kernel.  Then:
//   * k_csr_reduce / k_csr_scan_parts / k_csr_down: exclusive int64 prefix
//     scan of the counts -> offsets[0..M] (offsets[M] = number of edges);
//   * k_csr_gather: after the caller has allocated offsets[M] entries, copies
//     each unmarked row from the staging area to [offsets[i], offsets[i+1]);
//     the marked rows are written there by the selection kernel.
#include "frnn_host.h"

namespace frnn {

namespace {

constexpr int kCsrThreads = 1024;
constexpr int kCsrItems = 8;
constexpr int kCsrChunk = kCsrThreads * kCsrItems;

__device__ __forceinline__ int64_t row_count(const int32_t* cnt, int64_t i, int64_t M) {
    return i < M ? (int64_t)(cnt[i] & kCsrCountMask) : 0;
}

// exclusive scan of one value per thread over the block; returns the
// thread's exclusive prefix, *total gets the block's sum
__device__ int64_t block_scan64(int64_t v, int64_t* warp_tot, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int64_t w = warp_tot[lane];   // kCsrThreads / 32 == 32 warps
        int64_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        warp_tot[lane] = z - w;
        if (lane == 31) *total = z;
    }
    __syncthreads();
    const int64_t r = x - v + warp_tot[warp];
    __syncthreads();   // warp_tot is reused by the caller's next scan
    return r;
}

// per chunk of kCsrChunk counts: their sum
__global__ void __launch_bounds__(kCsrThreads) k_csr_reduce(const int32_t* cnt, int64_t M,
                                                            int64_t* parts) {
    pdl_trigger();
    pdl_wait();
    __shared__ int64_t red[kCsrThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kCsrChunk;
    int64_t s = 0;
    for (int k = 0; k < kCsrItems; ++k) s += row_count(cnt, base + (int64_t)k * kCsrThreads + threadIdx.x, M);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t t = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) parts[blockIdx.x] = t;
    }
}

// one block: exclusive scan of the nb chunk sums in place, walking them in
// blocks of kCsrThreads with a running carry
__global__ void __launch_bounds__(kCsrThreads) k_csr_scan_parts(int64_t* parts, int64_t nb) {
    pdl_trigger();
    pdl_wait();
    __shared__ int64_t warp_tot[kCsrThreads / 32];
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kCsrThreads) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? parts[i] : 0;
        const int64_t ex = block_scan64(v, warp_tot, &tot);
        if (i < nb) parts[i] = carry + ex;
        __syncthreads();
        carry += tot;
        __syncthreads();
    }
}

// offsets of one chunk: the chunk's exclusive scan plus its part's prefix;
// the last chunk also writes offsets[M]
__global__ void __launch_bounds__(kCsrThreads) k_csr_down(const int32_t* cnt, int64_t M,
                                                          const int64_t* parts, int64_t* offsets) {
    pdl_trigger();
    pdl_wait();
    __shared__ int64_t warp_tot[kCsrThreads / 32];
    __shared__ int64_t tot;
    const int64_t base = (int64_t)blockIdx.x * kCsrChunk + (int64_t)threadIdx.x * kCsrItems;
    int64_t v[kCsrItems];
    int64_t t = 0;
#pragma unroll
    for (int k = 0; k < kCsrItems; ++k) {
        v[k] = row_count(cnt, base + k, M);
        t += v[k];
    }
    int64_t ex = block_scan64(t, warp_tot, &tot) + (parts ? parts[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kCsrItems; ++k) {
        if (base + k < M) offsets[base + k] = ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        offsets[M] = tot + (parts ? parts[blockIdx.x] : 0);
}

// One warp per 32 consecutive rows.  Their entries are contiguous in the
// output ([offsets[r0], offsets[r0 + 32]) minus the rows the selection
// kernel writes), so the warp walks them as one flat range: entry t of the
// range belongs to the row whose exclusive prefix (within the 32) is the last
// one <= t (a binary search over the lanes' prefixes with shuffles); every
// lane copies one entry per step and the stores of a step are contiguous.
__global__ void __launch_bounds__(256) k_csr_gather(const int32_t* cnt, const int64_t* offsets,
                                                    const int32_t* sidx, const float* sd2,
                                                    int64_t M, int32_t* idx, float* dist2,
                                                    int64_t cap, int64_t row0, int64_t row1) {
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // rows [row0, row1) (row0 a multiple of 32)
    for (int64_t w = (row0 >> 5) + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
         w * 32 < row1; w += nw) {
        const int64_t r0 = w * 32;
        const int64_t i = r0 + lane;
        const int32_t c = i < row1 ? cnt[i] : 0;
        const int own = (c & kCsrSpill) ? 0 : c;   // spilled rows: written by the selection kernel
        int incl = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int excl = incl - own;
        const int T = __shfl_sync(0xffffffffu, incl, 31);
        const int64_t o_lane = i < row1 ? offsets[i] : 0;
        for (int base = 0; base < T; base += 32) {
            const int t = base + lane;
            int R = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int v = __shfl_sync(0xffffffffu, excl, R + st);
                if (v <= t) R += st;
            }
            const int e = t - __shfl_sync(0xffffffffu, excl, R);
            const int64_t dst = __shfl_sync(0xffffffffu, o_lane, R) + e;
            // cap: entries the output holds (a caller that gathers before
            // it knows the edge count passes its capacity; the call then
            // fails when the count exceeds it, and nothing past it is written)
            if (t < T && dst < cap) {
                const int64_t src = (r0 + R) * kCsrStageW + e;
                idx[dst] = sidx[src];
                dist2[dst] = sd2[src];
            }
        }
    }
}

}  // namespace

void enqueue_csr_offsets(const int32_t* cnt, int64_t M, int64_t* parts, int64_t* offsets,
                         cudaStream_t st) {
    const int64_t nb = std::max<int64_t>(1, ceil_div(M, kCsrChunk));
    if (nb > 1) {
        launch_pdl(k_csr_reduce, dim3((unsigned)nb), dim3(kCsrThreads), 0, st, cnt, M, parts);
        launch_pdl(k_csr_scan_parts, dim3(1), dim3(kCsrThreads), 0, st, parts, nb);
    }
    launch_pdl(k_csr_down, dim3((unsigned)nb), dim3(kCsrThreads), 0, st, cnt, M, nb > 1 ? parts : nullptr, offsets);
}

int64_t csr_parts_needed(int64_t M) { return std::max<int64_t>(1, ceil_div(M, kCsrChunk)); }

void enqueue_csr_gather(const int32_t* cnt, const int64_t* offsets, const int32_t* sidx,
                        const float* sd2, int64_t M, int32_t* idx, float* dist2, int num_sms,
                        cudaStream_t st, int64_t cap, int64_t row0, int64_t row1) {
    if (row1 < 0) row1 = M;
    if (row1 <= row0) return;
    const int64_t warps = ceil_div(row1 - row0, 32);
    const int64_t blocks = std::min<int64_t>(ceil_div(warps, 8), (int64_t)num_sms * 8);
    launch_pdl(k_csr_gather, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256), 0, st, cnt,
               offsets, sidx, sd2, M, idx, dist2, cap, row0, row1);
}

}  // namespace frnn
