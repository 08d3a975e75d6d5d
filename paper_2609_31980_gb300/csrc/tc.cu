// tc.cu — tensor-core path: a BF16 tcgen05 pre-filter over grid candidate
// tiles, followed by the exact float32 recheck of every survivor.
//
// The squared distance is written as n(x) + n(y) - 2 x.y, the dot products of
// a 128-query tile with a chunk of up to 256 candidates computed by one
// tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in tensor memory).
// The filter only has to be conservative: every pair the float32 contract
// accepts must pass it; each survivor is then recomputed with the exact
// contract, so results are bit-identical to the grid path and the oracle.
//
// Operands (per point, built once per grid by k_tc_prep):
//   x' = fl(x - c)             c = centre of the event's bounding box
//   hi = bf16(x'), lo = bf16(x' - hi)          (x' - hi is exact in float32)
//   query row  A = [hi, hi, lo, 1, 1, 0...]
//   candidate  B = [hi, lo, hi, m_hi, m_lo, 0...],  m = -n/2 split in two bf16,
//                  n = ||hi + lo||^2 in float32
// so acc = A.B ~= x'.y' - n(y)/2 and the pair passes when acc >= t(x) with
// t(x) = (n(x) - Theta)/2 rounded down.
//
// Margin (proof sketch; every factor below is a generous upper bound).  Let
// u = 2^-24, nu^2 the largest n over the event (queries and references).  The
// contract accepts => ||x - y||^2 <= R^2 = r2 (1 + 2^-18) (float32 partial
// sums of non-negative terms lose at most (1-u)^(2D+2) <= 1 - 2^-18 for
// D <= 16).  Centring moves a difference by <= u (|x'| + |y'|) per coordinate,
// the two-term split by <= 2^-16 |x'| (bf16 keeps 8 significant bits), so
// ||x^ - y^|| <= ||x - y|| + 2^-15 nu.  The GEMM drops lo.lo (<= 2^-16 nu^2),
// accumulates <= 3D + 2 exact bf16 products in float32 (<= 2^-17 (3 nu^2 + nu^2)
// with a 2x slack for the unspecified accumulation order), and the norms and
// m carry <= 2^-16 nu^2; all together |n(x) - 2 acc - ||x^ - y^||^2| <= 2^-13 nu^2.
// Theta = (R + 2^-14 nu)^2 + 2^-12 nu^2 therefore keeps every accepted pair.
// The margin is validated empirically by the parity tests (the tensor-core
// path's output must equal the oracle's bit for bit), and the tightest slack
// is what the false-candidate rate measures.
//
// Kernel organisation (one persistent CTA per SM, 8 warps, 512 TMEM columns):
//   * a producer warp issues cp.async.bulk copies of the A tile (128 query
//     rows) and, per chunk of up to 128 candidates, of the B tile plus the
//     float32 coordinates of the same candidates (for the recheck) into a
//     3-deep ring, and the MMAs (K/16 instructions per chunk) into one of two
//     TMEM accumulators (2 x 128 columns; two CTAs per SM share the 512);
//   * four epilogue warps: warp w reads TMEM lanes 32w.. with tcgen05.ld
//     32x32b.x32, tests 32 pairs per thread with a 3-input max tree, and where
//     a value reaches t(x) compacts the warp's survivors so that all 32 lanes
//     recheck them exactly from shared memory;
//   * per-query survivor lists in shared memory are sorted by (d2, index)
//     with a register network and written as coalesced rows.  Lists longer
//     than the capacity go to the exact selection kernel (query.cu).
// Every mbarrier wait is bounded; on a timeout the CTA records the status,
// stops, waits (bounded) for its copies and MMAs in flight and frees TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "frnn_host.h"

namespace frnn {

constexpr int kTcM = 128;        // queries per task = MMA M = TMEM lanes
constexpr int kTcN = 128;        // candidates per chunk = MMA N (multiple of 32)
constexpr int kTcAcc = 2;        // TMEM accumulators in flight (kTcAcc * kTcN = kTcCols)
constexpr int kTcEpi = 256;      // epilogue threads: warp w < 8 owns TMEM lanes 32 (w % 4)..
                                 // and column half w / 4 of every chunk
constexpr int kTcThreads = kTcEpi + 32;   // + one producer warp (bulk copies, MMA issue)
constexpr int kTcLStr = kTcM + 1;         // list table: one column per query row
constexpr int kTcMaxChunks = 128;         // chunk table entries kept in shared memory
constexpr int kTcMaxRows = kMaxNbrRows;   // neighbour rows per task
constexpr int kTcCols = 256;     // TMEM columns per CTA: two accumulators (2 CTAs / SM)
// (the producer warp is warp 4; epilogue warps 0..3 own the TMEM lane quarters)
constexpr int kTcList = 30;      // per-query survivor list capacity (2 CTAs / SM up to D = 12)
static_assert(kTcList <= kCsrStageW, "a staged compact row holds a whole list");

__host__ __device__ constexpr int tc_k_for(int D) { return ((3 * D + 2) + 15) / 16 * 16; }

// shared memory outside the operand ring
__host__ __device__ constexpr size_t tc_smem_fixed(int K, int DP);
// operand ring depth: as deep as fits two CTAs per SM (<= 110 KB each), 2..8
__host__ __device__ constexpr int tc_ring_for(int D);

constexpr int kTcSurvCap = 32 * 32;   // survivor (row, column) pairs of one warp and 32 columns

__host__ __device__ constexpr size_t tc_smem_fixed(int K, int DP) {
    return (size_t)kTcM * K * 2                                // A tile
           + (size_t)kTcList * kTcLStr * 8                     // per-query lists
           + (size_t)kTcM * DP * 4                             // query coordinates
           + (size_t)(kTcEpi / 32) * kTcSurvCap * 2;           // per-warp survivor buffers
}
__host__ __device__ constexpr size_t tc_slot_bytes(int K, int DP) {
    return (size_t)kTcN * K * 2 + (size_t)kTcN * DP * 4;       // B tile + float32 candidates
}
__host__ __device__ constexpr int tc_ring_for(int D) {
    int r = 8;
    while (r > 2 && tc_smem_fixed(tc_k_for(D), padded_dim(D)) +
                            (size_t)r * tc_slot_bytes(tc_k_for(D), padded_dim(D)) >
                        110 * 1024)
        --r;
    return r;
}
__host__ __device__ constexpr size_t tc_smem_bytes(int D) {
    return tc_smem_fixed(tc_k_for(D), padded_dim(D)) +
           (size_t)tc_ring_for(D) * tc_slot_bytes(tc_k_for(D), padded_dim(D));
}

// element offset of (row s, column k) in the core-matrix layout of rows of K
// bf16: groups of 8 rows, inside a group K/8 core matrices of 8 rows x 16 B
__device__ __forceinline__ int64_t cm_off(int64_t s, int k, int K) {
    return ((s >> 3) * (K >> 3) + (k >> 3)) * 64 + (s & 7) * 8 + (k & 7);
}

// ------------------------------------------------------------- operand prep

__device__ __forceinline__ int find_event_slot(const EventHdr* hdr, int E, int64_t s) {
    int lo = 0, hi = E - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (hdr[mid].pt_off <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint16_t bf16_bits(__nv_bfloat16 v) {
    return *reinterpret_cast<uint16_t*>(&v);
}

// One thread per slot: centred split operands, norm, per-event max norm.
// own: headers of this point set; ctr: headers whose centres to use.
template <int D>
__global__ void k_tc_prep(const EventHdr* own, const EventHdr* ctr, int E, int64_t n_total,
                          const float* pts, uint16_t* tcA, uint16_t* tcB, float* tcn,
                          int32_t* tcnu) {
    constexpr int K = tc_k_for(D);
    constexpr int DP = padded_dim(D);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_total) return;
    const int e = find_event_slot(own, E, s);
    const EventHdr& h = own[e];
    const bool real = s < h.pt_off + h.n && ctr[e].valid;
    uint16_t hi[D], lo[D];
    float n = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        hi[k] = 0;
        lo[k] = 0;
        if (real) {
            const float xc = __fsub_rn(pts[pt_index(s, k, DP)], ctr[e].ctr[k]);
            const __nv_bfloat16 bh = __float2bfloat16_rn(xc);
            const __nv_bfloat16 bl = __float2bfloat16_rn(__fsub_rn(xc, __bfloat162float(bh)));
            const float xh = __fadd_rn(__bfloat162float(bh), __bfloat162float(bl));
            n = __fmaf_rn(xh, xh, n);
            hi[k] = bf16_bits(bh);
            lo[k] = bf16_bits(bl);
        }
    }
    uint16_t one = 0, mh = 0, ml = 0;
    if (real) {
        const float mneg = -0.5f * n;
        const __nv_bfloat16 bmh = __float2bfloat16_rn(mneg);
        const __nv_bfloat16 bml = __float2bfloat16_rn(__fsub_rn(mneg, __bfloat162float(bmh)));
        one = bf16_bits(__float2bfloat16_rn(1.f));
        mh = bf16_bits(bmh);
        ml = bf16_bits(bml);
    }
    // A = [hi, hi, lo, 1, 1, 0...], B = [hi, lo, hi, m_hi, m_lo, 0...]
    auto a_el = [&](int j) -> uint32_t {
        return j < D ? hi[j] : j < 2 * D ? hi[j - D] : j < 3 * D ? lo[j - 2 * D]
               : (j == 3 * D || j == 3 * D + 1) ? one : 0;
    };
    auto b_el = [&](int j) -> uint32_t {
        return j < D ? hi[j] : j < 2 * D ? lo[j - D] : j < 3 * D ? hi[j - 2 * D]
               : j == 3 * D ? mh : j == 3 * D + 1 ? ml : 0;
    };
#pragma unroll
    for (int kg = 0; kg < K / 8; ++kg) {
        uint4 va, vb;
        va.x = a_el(8 * kg + 0) | (a_el(8 * kg + 1) << 16);
        va.y = a_el(8 * kg + 2) | (a_el(8 * kg + 3) << 16);
        va.z = a_el(8 * kg + 4) | (a_el(8 * kg + 5) << 16);
        va.w = a_el(8 * kg + 6) | (a_el(8 * kg + 7) << 16);
        vb.x = b_el(8 * kg + 0) | (b_el(8 * kg + 1) << 16);
        vb.y = b_el(8 * kg + 2) | (b_el(8 * kg + 3) << 16);
        vb.z = b_el(8 * kg + 4) | (b_el(8 * kg + 5) << 16);
        vb.w = b_el(8 * kg + 6) | (b_el(8 * kg + 7) << 16);
        const int64_t off = cm_off(s, 8 * kg, K);
        *reinterpret_cast<uint4*>(tcA + off) = va;
        *reinterpret_cast<uint4*>(tcB + off) = vb;
    }
    tcn[s] = n;
    // per-event maximum: reduce across the warp first when its lanes share an
    // event (almost always), one atomic per warp instead of one per point
    const int32_t on = real ? float_to_ordered(n) : INT32_MIN;
    const unsigned same = __match_any_sync(__activemask(), e);
    const int32_t wmax = __reduce_max_sync(same, on);
    if (real && (threadIdx.x & 31) == __ffs(same) - 1) atomicMax(tcnu + e, wmax);
}

// ------------------------------------------------------------- tcgen05 helpers

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05; no swizzle, base offset 0
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = n
__device__ __forceinline__ uint32_t mma_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// tcgen05.ld of 32 columns without the wait (several loads share one wait)
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

struct TcArgs {
    const EventHdr* ev;       // reference grid headers
    const Task* tasks;        // 128-query tasks of the query set
    const int32_t* ntasks;
    const uint16_t* tcA;      // query-set operands
    const uint16_t* tcB;      // reference operands
    const float* qn;          // query norms
    const int32_t* nu_q;      // per-event max norms (ordered ints)
    const int32_t* nu_r;
    const float* qpts;
    const int32_t* qperm;
    const int32_t* qcell;
    const float* rpts;
    const int32_t* rperm;
    const int32_t* cstart;
    int32_t* counts;          // single-event outputs or NULL (per-event headers)
    int32_t* idx;
    float* dist2;
    float r2;
    int32_t K;
    int32_t self;
    int32_t D;
    int32_t* task_counter;
    int32_t* status;
    Overflow* ovf;
    int32_t* ovf_count;
    int32_t ovf_cap;
    int32_t path_filter;                  // -1: every event; else only events with this path
    unsigned long long* stat_survivors;   // pre-filter survivors (false-candidate rate)
    unsigned long long* stat_accepted;    // exact accepts
    int32_t csr;                          // compact output: staging rows (see QueryArgs)
    int32_t* degree;
};

// Chunk geometry of a task: neighbour row L covers slot range [rs, re); its
// operand rows start at b8 = rs rounded down to 8 and end at e8 = re rounded
// up to 8; chunks of up to 256 rows (the MMA N, rounded up to 16).
struct ChunkTab {
    int rs[kTcMaxRows], re[kTcMaxRows], b8[kTcMaxRows], pref[kTcMaxRows + 1];
    int nrows, nch;
    int4 chunk[kTcMaxChunks];   // (start, n, lo, hi) of the first chunks
};

__device__ __forceinline__ void chunk_info_slow(const ChunkTab& t, int c, int& start, int& n,
                                                int& lo, int& hi) {
    int L = 0;
    while (L + 1 < t.nrows && t.pref[L + 1] <= c) ++L;
    start = t.b8[L] + (c - t.pref[L]) * kTcN;
    const int e8 = (t.re[L] + 7) & ~7;
    n = min(kTcN, e8 - start);
    n = (n + 31) & ~31;   // whole 32-column TMEM loads; extra rows are masked by [lo, hi)
    lo = t.rs[L];
    hi = t.re[L];
}

__device__ __forceinline__ void chunk_info(const ChunkTab& t, int c, int& start, int& n, int& lo,
                                           int& hi) {
    if (c < kTcMaxChunks) {
        const int4 v = t.chunk[c];
        start = v.x;
        n = v.y;
        lo = v.z;
        hi = v.w;
    } else {
        chunk_info_slow(t, c, start, n, lo, hi);
    }
}

template <int D>
__global__ void __launch_bounds__(kTcThreads, 2) k_tc_query(TcArgs a) {
    constexpr int K = tc_k_for(D);
    constexpr int KS = K / 16;
    constexpr int DP = padded_dim(D);
    constexpr int kTcRing = tc_ring_for(D);
    extern __shared__ __align__(1024) unsigned char smem[];
    uint16_t* As = reinterpret_cast<uint16_t*>(smem);
    uint16_t* Bs = As + kTcM * K;
    float* Fs = reinterpret_cast<float*>(Bs + kTcRing * kTcN * K);
    float* Ld = Fs + kTcRing * kTcN * DP;
    int32_t* Li = reinterpret_cast<int32_t*>(Ld + kTcList * kTcLStr);
    float* Qs = reinterpret_cast<float*>(Li + kTcList * kTcLStr);      // [128][DP]
    uint16_t* Sv = reinterpret_cast<uint16_t*>(Qs + kTcM * DP);        // [4][kTcSurvCap]

    // bar_b: chunk operands landed; bar_mma: accumulator ready; bar_acc:
    // epilogue done with an accumulator; bar_slot: epilogue done with a ring slot
    __shared__ __align__(8) uint64_t bar_a, bar_b[kTcRing], bar_mma[kTcAcc], bar_acc[kTcAcc],
        bar_slot[kTcRing];
    __shared__ uint32_t s_taddr;
    __shared__ Task s_task;
    __shared__ int s_done, s_abort;
    __shared__ ChunkTab s_ct;
    __shared__ int s_cnt[kTcM];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == kTcEpi / 32;
    const int half = (warp >> 2) & 1;          // column half of the chunk (epilogue warps)
    const int row = 32 * (warp & 3) + lane;    // TMEM lane / query row

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_taddr)), "n"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar_a, 1);
        for (int i = 0; i < kTcRing; ++i) {
            mbar_init(&bar_b[i], 1);
            mbar_init(&bar_slot[i], kTcEpi);   // every epilogue thread, every chunk
        }
        for (int i = 0; i < kTcAcc; ++i) {
            mbar_init(&bar_mma[i], 1);
            mbar_init(&bar_acc[i], kTcEpi);
        }
        s_abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;

    const uint32_t sA = smem_u32(As);
    const uint32_t sB = smem_u32(Bs);
    const uint32_t lbo = 128, sbo = (uint32_t)K * 16;
    const float r2 = a.r2;
    const int Kout = a.K;
    const int ntasks = *a.ntasks;

    uint32_t task_no = 0;
    uint32_t g0 = 0;          // global chunk counter at the start of the task
    unsigned long long n_surv = 0, n_acc = 0;

    auto abort_now = [&]() {
        atomicOr(a.status, kStatusTimeout);
        atomicExch(&s_abort, 1);
    };
    auto aborted = [&]() -> int { return *reinterpret_cast<volatile int*>(&s_abort); };

    for (;;) {
        __syncthreads();
        if (tid == kTcEpi) {
            const int t = atomicAdd(a.task_counter, 1);
            s_done = (t >= ntasks) || aborted();
            if (t < ntasks) s_task = a.tasks[t];
        }
        __syncthreads();
        if (s_done) break;
        const Task tk = s_task;
        const EventHdr& h = a.ev[tk.ev];
        if (a.path_filter >= 0 && h.path != a.path_filter) continue;   // another launch's event
        int32_t* counts = a.counts ? a.counts : h.counts;
        int32_t* oidx = a.counts ? a.idx : h.idx;
        float* od2 = a.counts ? a.dist2 : h.dist2;
        const int w0 = tk.qslot & ~7;
        const int qs = w0 + row;
        const bool active = !producer && qs >= tk.qslot && qs < tk.qslot + tk.nq;
        const int qorig = active ? a.qperm[qs] : 0;
        if (!h.valid) {
            // grid built from non-finite input: empty rows (frnn_sync reports it)
            if (active) {
                for (int e = 0; e < Kout && !a.csr; ++e) {
                    oidx[(int64_t)qorig * Kout + e] = -1;
                    od2[(int64_t)qorig * Kout + e] = INFINITY;
                }
                counts[qorig] = 0;
                if (a.degree) a.degree[qorig] = 0;
            }
            continue;
        }
        if (producer) {
            // neighbour rows and chunk table
            const int dims0 = h.dims[0], m = h.m;
            const int xa = a.qcell[tk.qslot] % dims0;
            const int xb = a.qcell[tk.qslot + tk.nq - 1] % dims0;
            // (2m+1)^(naxes-1) <= kTcMaxRows rows (the grid parameters ensure
            // it), 32 per round with a running chunk count
            const int nrows = neighbour_rows(h);
            int carry = 0;
            for (int rr = 0; rr * 32 < nrows; ++rr) {
                const int l = rr * 32 + lane;
                int rs = 0, re = 0;
                int64_t rowbase;
                if (l < nrows && neighbour_row(h, tk.row, l, rowbase)) {
                    rs = a.cstart[rowbase + max(xa - m, 0)];
                    re = a.cstart[rowbase + min(xb + m, dims0 - 1) + 1];
                }
                const int b8 = rs & ~7;
                const int e8 = (re + 7) & ~7;
                const int nch = re > rs ? (e8 - b8 + kTcN - 1) / kTcN : 0;
                int pre = nch;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += v;
                }
                if (l < kTcMaxRows) {
                    s_ct.rs[l] = rs;
                    s_ct.re[l] = re;
                    s_ct.b8[l] = b8;
                    s_ct.pref[l] = carry + pre - nch;
                }
                // this lane's row: its chunks' (start, n, lo, hi)
                for (int j = 0; j < nch; ++j) {
                    const int c = carry + pre - nch + j;
                    if (c >= kTcMaxChunks) break;
                    const int start = b8 + j * kTcN;
                    int n = min(kTcN, e8 - start);
                    n = (n + 31) & ~31;
                    s_ct.chunk[c] = make_int4(start, n, rs, re);
                }
                carry += __shfl_sync(0xffffffffu, pre, 31);
            }
            if (lane == 0) {
                s_ct.nch = carry;
                s_ct.nrows = nrows;
            }
        } else if (half == 0) {
            // this thread's query: float32 coordinates (shared: the recheck
            // reads them from any lane)
#pragma unroll
            for (int k = 0; k < D; ++k)
                Qs[row * DP + k] = active ? a.qpts[pt_index(qs, k, DP)] : 0.f;
            s_cnt[row] = 0;
        }
        __syncthreads();
        const int nch = s_ct.nch;

        if (producer) {
            // ---------------------------------------------------- producer
            if (lane == 0 && nch > 0) {
                // ring slot g % R is free once the epilogue of chunk g - R is done
                auto slot_free_now = [&](uint32_t g) -> bool {
                    if (g < (uint32_t)kTcRing) return true;
                    uint32_t ok2;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                        "selp.u32 %0, 1, 0, p;\n\t}"
                        : "=r"(ok2)
                        : "r"(smem_u32(&bar_slot[g % kTcRing])),
                          "r"(((g - kTcRing) / kTcRing) & 1u)
                        : "memory");
                    return ok2 != 0;
                };
                auto issue_load = [&](int c, uint32_t g) {
                    int start, n, lo, hi;
                    chunk_info(s_ct, c, start, n, lo, hi);
                    const int slot = g % kTcRing;
                    const uint32_t bB = (uint32_t)n * K * 2;
                    const uint32_t bF = (uint32_t)n * DP * 4;
                    mbar_arrive_expect_tx(&bar_b[slot], bB + bF);
                    bulk_g2s(Bs + (size_t)slot * kTcN * K, a.tcB + cm_off(start, 0, K), bB,
                             &bar_b[slot]);
                    bulk_g2s(Fs + (size_t)slot * kTcN * DP, a.rpts + (int64_t)start * DP, bF,
                             &bar_b[slot]);
                };
                const uint32_t bA = (uint32_t)kTcM * K * 2;
                mbar_arrive_expect_tx(&bar_a, bA);
                bulk_g2s(As, a.tcA + cm_off(w0, 0, K), bA, &bar_a);
                int next_load = 0, issued_mma = 0;
                bool ok = true;
                // loads run ahead as far as ring slots are free
                while (next_load < nch && next_load < kTcRing && slot_free_now(g0 + next_load)) {
                    issue_load(next_load, g0 + next_load);
                    ++next_load;
                }
                ok = mbar_wait_bounded(&bar_a, task_no & 1u);
                for (int c = 0; ok && c < nch; ++c) {
                    const uint32_t g = g0 + c;
                    const int slot = g % kTcRing;
                    while (ok && next_load <= c) {   // this chunk's operands must be on their way
                        const uint32_t gl = g0 + next_load;
                        if (gl >= (uint32_t)kTcRing)
                            ok = mbar_wait_bounded(&bar_slot[gl % kTcRing],
                                                   ((gl - kTcRing) / kTcRing) & 1u);
                        if (ok) {
                            issue_load(next_load, gl);
                            ++next_load;
                        }
                    }
                    // operands landed and the accumulator's previous epilogue done
                    if (ok) ok = mbar_wait_bounded(&bar_b[slot], (g / kTcRing) & 1u);
                    if (ok && g >= (uint32_t)kTcAcc)
                        ok = mbar_wait_bounded(&bar_acc[g % kTcAcc], ((g - kTcAcc) / kTcAcc) & 1u);
                    if (!ok) break;
                    tc_fence_after();
                    int start, n, lo, hi;
                    chunk_info(s_ct, c, start, n, lo, hi);
                    const uint32_t idesc = mma_idesc(n);
                    const uint32_t bbase = sB + (uint32_t)(slot * kTcN * K * 2);
#pragma unroll
                    for (int ks = 0; ks < KS; ++ks) {
                        mma_bf16(taddr + (g % kTcAcc) * kTcN, smem_desc(sA + ks * 256, lbo, sbo),
                                 smem_desc(bbase + ks * 256, lbo, sbo), idesc, ks > 0 ? 1u : 0u);
                    }
                    mma_commit(&bar_mma[g % kTcAcc]);
                    issued_mma = c + 1;
                    while (next_load < nch && next_load < c + 1 + kTcRing &&
                           slot_free_now(g0 + next_load)) {
                        issue_load(next_load, g0 + next_load);
                        ++next_load;
                    }
                }
                if (!ok) {
                    abort_now();
                    // wait (bounded) for the copies and MMAs in flight
                    for (int c = issued_mma; c < next_load; ++c)
                        mbar_wait_bounded(&bar_b[(g0 + c) % kTcRing], ((g0 + c) / kTcRing) & 1u);
                    if (issued_mma > 0)
                        mbar_wait_bounded(&bar_mma[(g0 + issued_mma - 1) % kTcAcc],
                                          ((g0 + issued_mma - 1) / kTcAcc) & 1u);
                }
            }
            __syncwarp();
        } else {
            // ---------------------------------------------------- epilogue
            float tx = INFINITY;
            if (active) {
                const double nu2 = fmax((double)ordered_to_float(a.nu_q[tk.ev]),
                                        (double)ordered_to_float(a.nu_r[tk.ev]));
                const double nu = sqrt(fmax(nu2, 0.0));
                const double R = sqrt((double)r2 * (1.0 + 0x1p-18));
                const double th = (R + 0x1p-14 * nu) * (R + 0x1p-14 * nu) + 0x1p-12 * nu2;
                tx = __double2float_rd(((double)a.qn[qs] - th) * 0.5);
            }
            const int self_slot = a.self ? qs : -1;
            uint16_t* sv = Sv + warp * kTcSurvCap;
            for (int c = 0; c < nch; ++c) {
                const uint32_t g = g0 + c;
                // accumulator ready and the chunk's staged coordinates visible
                if (!aborted()) {
                    if (!mbar_wait_bounded(&bar_mma[g % kTcAcc], (g / kTcAcc) & 1u) ||
                        !mbar_wait_bounded(&bar_b[g % kTcRing], (g / kTcRing) & 1u))
                        abort_now();
                }
                __syncwarp();
                tc_fence_after();
                if (!__shfl_sync(0xffffffffu, aborted(), 0)) {
                    int start, n, lo, hi;
                    chunk_info(s_ct, c, start, n, lo, hi);
                    const float* F = Fs + (size_t)(g % kTcRing) * kTcN * DP;
                    const uint32_t tbase =
                        taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (g % kTcAcc) * kTcN;
                    const int cend = min(n, kTcN / 2 * (half + 1));
#pragma unroll 1
                    for (int col0 = kTcN / 2 * half; col0 < cend; col0 += 32) {   // n: multiple of 32
                        float v[32];
                        __syncwarp();
                        tmem_ld32(tbase + col0, v);
                        float mx = fmax3(v[0], v[1], v[2]);
#pragma unroll
                        for (int j = 3; j < 31; j += 2) mx = fmax3(mx, v[j], v[j + 1]);
                        mx = fmaxf(mx, v[31]);
                        if (!__any_sync(0xffffffffu, mx >= tx)) continue;
                        // columns of this group inside the chunk's own row range
                        const int c0 = start + col0;
                        const int jlo = max(lo - c0, 0), jhi = min(hi - c0, 32);
                        uint32_t valid =
                            jhi > jlo ? (((jhi - jlo) == 32 ? 0xffffffffu
                                                            : ((1u << (jhi - jlo)) - 1u))
                                         << jlo)
                                      : 0u;
                        if (self_slot >= c0 && self_slot < c0 + 32)
                            valid &= ~(1u << (self_slot - c0));
                        uint32_t mask = 0;
                        if (mx >= tx) {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (v[j] >= tx) mask |= 1u << j;
                            mask &= valid;
                        }
                        // compact the warp's (row, column) survivors, then
                        // recheck them with all 32 lanes
                        const int nb = __popc(mask);
                        int off = nb;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int t2 = __shfl_up_sync(0xffffffffu, off, o);
                            if (lane >= o) off += t2;
                        }
                        const int total = __shfl_sync(0xffffffffu, off, 31);
                        off -= nb;
                        while (mask) {
                            const int j = __ffs(mask) - 1;
                            mask &= mask - 1;
                            sv[off++] = (uint16_t)((lane << 5) | j);
                        }
                        __syncwarp();
                        n_surv += (lane == 0) ? total : 0;
                        for (int b = 0; b < total; b += 32) {
                            if (b + lane < total) {
                                const int pr = sv[b + lane];
                                const int r = 32 * (warp & 3) + (pr >> 5);
                                const int cs = c0 + (pr & 31);
                                // exact contract from the staged float32 coordinates
                                const float* f = F + (size_t)(cs - start) * DP;
                                const float* qv = Qs + r * DP;
                                float sd = 0.f;
#pragma unroll
                                for (int k = 0; k < D; ++k) {
                                    const float d = __fsub_rn(qv[k], f[k]);
                                    sd = __fadd_rn(sd, __fmul_rn(d, d));
                                }
                                if (sd <= r2) {
                                    ++n_acc;
                                    const int pos = atomicAdd(&s_cnt[r], 1);
                                    if (pos < kTcList) {   // original index looked up here
                                        Ld[pos * kTcLStr + r] = sd;
                                        Li[pos * kTcLStr + r] = a.rperm[cs];
                                    }
                                }
                            }
                        }
                        __syncwarp();
                    }
                }
                tc_fence_before();
                mbar_arrive(&bar_acc[g % kTcAcc]);
                mbar_arrive(&bar_slot[g % kTcRing]);
            }
        }
        __syncthreads();
        if (aborted()) break;
        g0 += nch;
        if (nch > 0) ++task_no;
        if (producer) continue;

        // every query sorts its own list by (d2, original index), all threads
        // in parallel (register bitonic network, see sort_list)
        const int cnt = s_cnt[row];
        const bool spill = active && cnt > kTcList;
        if (half == 0) {
            sort_list(Ld + row, Li + row, kTcLStr, (active && !spill) ? cnt : 0, nullptr);
            if (active && !spill) counts[qorig] = min(cnt, Kout);
            if (active && spill && a.csr) counts[qorig] = kCsrSpill;   // counted by the selection kernel
            if (active && !spill && a.degree) a.degree[qorig] = cnt;
        }
        if (spill && half == 0) {
            // longer than the list: the exact selection kernel finishes this row
            const int pos = atomicAdd(a.ovf_count, 1);
            if (pos < a.ovf_cap) {
                a.ovf[pos].qslot = qs;
                a.ovf[pos].ev = tk.ev;
            } else {
                atomicOr(a.status, kStatusCapacity);
            }
        }
        // rows sorted by the half-0 threads; then coalesced row writes, each
        // epilogue warp 16 of the 128 rows
        asm volatile("bar.sync 1, %0;" ::"n"(kTcEpi) : "memory");
        const unsigned skip = __ballot_sync(0xffffffffu, !active || spill);   // rows 32(w%4)..
        for (int qq = 0; qq < 16; ++qq) {
            const int ql = 16 * half + qq;                 // lane of this row in the warp
            if (skip & (1u << ql)) continue;
            const int r = 32 * (warp & 3) + ql;
            const int c = min(__shfl_sync(0xffffffffu, cnt, ql), Kout);
            const int qo = __shfl_sync(0xffffffffu, qorig, ql);
            const int rstride = a.csr ? kCsrStageW : Kout;   // compact: staging row, no padding
            int32_t* irow = oidx + (int64_t)qo * rstride;
            float* drow = od2 + (int64_t)qo * rstride;
            for (int e = lane; e < (a.csr ? c : Kout); e += 32) {
                const bool real = e < c;
                irow[e] = real ? Li[e * kTcLStr + r] : -1;
                drow[e] = real ? Ld[e * kTcLStr + r] : INFINITY;
            }
        }
    }
    if (a.stat_survivors && !producer) {
        atomicAdd(a.stat_survivors, n_surv);
        atomicAdd(a.stat_accepted, n_acc);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "n"(kTcCols)
                     : "memory");
    }
}

// ------------------------------------------------------------- host

void tc_free(GridBufs& g) {
    if (g.tc_base) cudaFree(g.tc_base);
    g.tc_base = nullptr;
    g.tc_bytes = 0;
    g.tc_cap_rows = g.tc_cap_tasks = g.tc_cap_E = g.tc_cap_L = 0;
    g.tc_rtask = nullptr;
    g.rtask = nullptr;
    g.tc_ready = false;
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Allocate (or keep) the operand buffers of a point set; enqueues nothing but
// the one-time zeroing of a fresh allocation (on the legacy default stream,
// synchronised, so it may run before a capture begins).
frnn_status tc_reserve(GridBufs& g, std::string& err) {
    const int K = tc_k_for(g.D);
    const int64_t rows = (g.n_total + 7) / 8 * 8 + kTcRowPad;
    // a tile never spans two rows of cells and only rows holding a point open
    // one: a row of c queries takes at most floor(c / 128) + 1 tiles, or + 2
    // when its start alignment (up to 7 slots) carries it past a multiple of
    // 128, which needs c >= 121; so per event at most n / 128 + rows + n / 121
    int64_t tcap = 0;
    for (int e = 0; e < g.E; ++e)
        tcap += g.h_hdr[e].n / kTcM + g.h_hdr[e].n / 64 +
                std::min<int64_t>(g.h_hdr[e].cell_cap, g.h_hdr[e].n) + 2;
    if (tcap >= INT32_MAX) {
        err = "too many tensor-core tiles for one call";
        return FRNN_ERR_INVALID_ARG;
    }
    if (g.tc_base && g.tc_K == K && g.tc_cap_rows >= rows && g.tc_cap_tasks >= tcap &&
        g.tc_cap_E >= g.E && g.tc_cap_L >= g.L) {
        g.rtask = g.tc_rtask;
        return FRNN_OK;
    }
    tc_free(g);
    const size_t bA = al256(sizeof(uint16_t) * rows * K);
    const size_t bn = al256(sizeof(float) * rows);
    const size_t bnu = al256(sizeof(int32_t) * std::max(g.E, 1));
    const size_t bt = al256(sizeof(Task) * tcap);
    const size_t brt = al256(sizeof(int32_t) * std::max<int64_t>(g.L, 1));
    void* base = nullptr;
    cudaError_t ce = cudaMalloc(&base, 2 * bA + bn + bnu + bt + brt + 256);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        err = "cudaMalloc of tensor-core operands failed";
        return FRNN_ERR_OUT_OF_MEMORY;
    }
    char* b = static_cast<char*>(base);
    g.tc_base = base;
    g.tc_bytes = 2 * bA + bn + bnu + bt + brt + 256;
    g.tcA = reinterpret_cast<uint16_t*>(b);
    g.tcB = reinterpret_cast<uint16_t*>(b + bA);
    g.tcn = reinterpret_cast<float*>(b + 2 * bA);
    g.tcnu = reinterpret_cast<int32_t*>(b + 2 * bA + bn);
    g.tc_tasks = reinterpret_cast<Task*>(b + 2 * bA + bn + bnu);
    g.tc_rtask = reinterpret_cast<int32_t*>(b + 2 * bA + bn + bnu + bt);
    g.rtask = g.tc_rtask;   // scratch of the task builder (per row of cells)
    g.tc_cap_L = g.L;
    g.tc_cap_rows = rows;
    g.tc_cap_tasks = tcap;
    g.tc_cap_E = g.E;
    g.tc_K = K;
    // rows past the last slot stay zero (chunks may read them)
    ce = cudaMemset(base, 0, 2 * bA + bn);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        err = "zeroing tensor-core operands failed";
        return FRNN_ERR_CUDA;
    }
    return FRNN_OK;
}

frnn_status tc_prepare(GridBufs& g, const GridBufs& center_src, int32_t* d_status,
                       cudaStream_t st, std::string& err, int path_filter, int64_t i0,
                       int64_t i1) {
    frnn_status s0 = tc_reserve(g, err);
    if (s0 != FRNN_OK) return s0;
    const int K = tc_k_for(g.D);
    cudaMemsetAsync(g.tcnu, 0, sizeof(int32_t) * g.E, st);   // ordered(0.0f) == 0
    if (g.n_total > 0) {
        const unsigned nb = (unsigned)ceil_div(g.n_total, 128);
        switch (g.D) {
#define FRNN_PREP(d)                                                                         \
    case d:                                                                                  \
        k_tc_prep<d><<<nb, 128, 0, st>>>(g.hdr, center_src.hdr, g.E, g.n_total, g.pts, g.tcA, \
                                         g.tcB, g.tcn, g.tcnu);                              \
        break;
            FRNN_PREP(8) FRNN_PREP(9) FRNN_PREP(10) FRNN_PREP(11) FRNN_PREP(12)
            FRNN_PREP(13) FRNN_PREP(14) FRNN_PREP(15) FRNN_PREP(16)
#undef FRNN_PREP
            default:
                err = "tensor-core path needs 8 <= D <= 16";
                return FRNN_ERR_UNSUPPORTED;
        }
        (void)K;
    }
    enqueue_tasks(g, kTcM, 8, g.tc_tasks, g.tc_cap_tasks, g.scalars + kScTcTasks, d_status, st,
                  path_filter, i0, i1);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("tensor-core prep launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    g.tc_ready = true;
    return FRNN_OK;
}

frnn_status enqueue_tc_query(const QueryLaunch& q, cudaStream_t st, std::string& err) {
    const GridBufs& qs = *q.qset;
    const GridBufs& rs = *q.rset;
    const int D = rs.D;
    const int K = tc_k_for(D);
    TcArgs a{};
    a.ev = rs.hdr;
    a.tasks = qs.tc_tasks;
    a.ntasks = qs.scalars + kScTcTasks;
    a.tcA = qs.tcA;
    a.tcB = rs.tcB;
    a.qn = qs.tcn;
    a.nu_q = qs.tcnu;
    a.nu_r = rs.tcnu;
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
    a.D = D;
    a.task_counter = qs.scalars + kScTcCounter;
    a.status = q.d_status;
    a.ovf = qs.ovf;
    a.ovf_count = qs.scalars + kScOvfCount;
    a.ovf_cap = (int32_t)std::max<int64_t>(qs.n_total, 1);
    a.path_filter = q.path_filter;
    a.stat_survivors = q.tc_stats;
    a.stat_accepted = q.tc_stats ? q.tc_stats + 1 : nullptr;
    a.csr = q.csr;
    a.degree = q.degree;
    cudaMemsetAsync(qs.scalars + kScOvfCount, 0, sizeof(int32_t), st);
    cudaMemsetAsync(qs.scalars + kScTcCounter, 0, sizeof(int32_t), st);
    if (q.kev[0]) cudaEventRecord(q.kev[0], st);
    cudaError_t ce = cudaSuccess;
    auto launch = [&](auto kern, size_t smem) {
        ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ce == cudaSuccess) {
            kern<<<2 * q.num_sms, kTcThreads, smem, st>>>(a);
            ce = cudaGetLastError();
        }
    };
    switch (D) {
        case 8: launch(k_tc_query<8>, tc_smem_bytes(8)); break;
        case 9: launch(k_tc_query<9>, tc_smem_bytes(9)); break;
        case 10: launch(k_tc_query<10>, tc_smem_bytes(10)); break;
        case 11: launch(k_tc_query<11>, tc_smem_bytes(11)); break;
        case 12: launch(k_tc_query<12>, tc_smem_bytes(12)); break;
        case 13: launch(k_tc_query<13>, tc_smem_bytes(13)); break;
        case 14: launch(k_tc_query<14>, tc_smem_bytes(14)); break;
        case 15: launch(k_tc_query<15>, tc_smem_bytes(15)); break;
        case 16: launch(k_tc_query<16>, tc_smem_bytes(16)); break;
        default:
            err = "tensor-core path needs 8 <= D <= 16";
            return FRNN_ERR_UNSUPPORTED;
    }
    if (ce != cudaSuccess) {
        err = std::string("tensor-core query launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
    if (q.kev[1]) cudaEventRecord(q.kev[1], st);
    // rows whose lists overflowed: exact selection kernel
    QueryArgs o{};
    o.ev = rs.hdr;
    o.qpts = qs.pts;
    o.qperm = qs.perm;
    o.qcell = qs.cell;
    o.rpts = rs.pts;
    o.rperm = rs.perm;
    o.cstart = rs.cstart;
    o.counts = q.counts;
    o.idx = q.idx;
    o.dist2 = q.dist2;
    o.r2 = q.r2;
    o.K = q.K;
    o.self = q.self;
    o.D = D;
    o.status = q.d_status;
    o.ovf = qs.ovf;
    o.ovf_count = qs.scalars + kScOvfCount;
    o.ovf_cap = a.ovf_cap;
    o.path_filter = -1;   // the list only holds rows this launch queued
    o.csr = q.csr;
    o.ovf_mode = q.ovf_mode;
    o.degree = q.degree;
    o.row_off = q.row_off;
    return enqueue_overflow(o, q.num_sms, st, err);
}

}  // namespace frnn
