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
//   * thread 0 is the producer: cp.async.bulk of the A tile (128 query rows)
//     and, per chunk, of the B tile plus the float32 coordinates of the same
//     candidates (for the recheck) into a 3-deep ring, then issues the MMAs
//     (K/16 instructions, accumulator double-buffered in TMEM: 2 x 256 cols);
//   * all 8 warps run the epilogue: warp w reads TMEM lanes 32 (w % 4).. and
//     column half w / 4 with tcgen05.ld 32x32b.x32, tests 32 pairs with a
//     3-input max tree, and only where a value reaches t(x) builds the bit
//     mask and rechecks those candidates exactly from shared memory;
//   * per (query, half) survivor lists in shared memory are merged, sorted by
//     (d2, index) per query and written as coalesced rows.  Lists longer than
//     the capacity go to the exact selection kernel (query.cu).
// Every mbarrier wait is bounded; on a timeout the CTA records the status,
// stops, waits (bounded) for its copies and MMAs in flight and frees TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "frnn_host.h"

namespace frnn {

constexpr int kTcM = 128;        // queries per task = MMA M = TMEM lanes
constexpr int kTcN = 256;        // candidates per chunk = max MMA N
constexpr int kTcThreads = 256;  // 8 warps
constexpr int kTcLStr = kTcThreads + 1;
constexpr int kTcMaxRows = 32;   // neighbour rows per task (m <= 2)
constexpr int kTcRing = 3;       // operand ring depth

__host__ __device__ constexpr int tc_k_for(int D) { return ((3 * D + 2) + 15) / 16 * 16; }
__host__ __device__ constexpr int tc_list_cap(int KS) { return KS >= 4 ? 30 : 32; }

__host__ __device__ constexpr size_t tc_smem_bytes(int KS, int DP) {
    return (size_t)kTcM * 16 * KS * 2                          // A tile
           + (size_t)kTcRing * kTcN * 16 * KS * 2              // B ring
           + (size_t)kTcRing * kTcN * DP * 4                   // float32 candidate ring
           + (size_t)tc_list_cap(KS) * kTcLStr * 8;            // per-thread lists
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
__global__ void k_tc_prep(const EventHdr* own, const EventHdr* ctr, int E, int D, int64_t n_total,
                          const float* pts, uint16_t* tcA, uint16_t* tcB, float* tcn,
                          int32_t* tcnu, int K) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_total) return;
    const int e = find_event_slot(own, E, s);
    const EventHdr& h = own[e];
    const bool real = s < h.pt_off + h.n && ctr[e].valid;
    const int DP = padded_dim(D);
    uint16_t ra[64], rb[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) { ra[k] = 0; rb[k] = 0; }
    float n = 0.f;
    if (real) {
        const __nv_bfloat16 one = __float2bfloat16_rn(1.f);
#pragma unroll
        for (int k = 0; k < kMaxD; ++k) {
            if (k < D) {
                const float xc = __fsub_rn(pts[pair_index(s, k, DP)], ctr[e].ctr[k]);
                const __nv_bfloat16 hi = __float2bfloat16_rn(xc);
                const __nv_bfloat16 lo = __float2bfloat16_rn(__fsub_rn(xc, __bfloat162float(hi)));
                const float xh = __fadd_rn(__bfloat162float(hi), __bfloat162float(lo));
                n = __fmaf_rn(xh, xh, n);
                ra[k] = bf16_bits(hi); ra[D + k] = bf16_bits(hi); ra[2 * D + k] = bf16_bits(lo);
                rb[k] = bf16_bits(hi); rb[D + k] = bf16_bits(lo); rb[2 * D + k] = bf16_bits(hi);
            }
        }
        const float mneg = -0.5f * n;
        const __nv_bfloat16 mh = __float2bfloat16_rn(mneg);
        const __nv_bfloat16 ml = __float2bfloat16_rn(__fsub_rn(mneg, __bfloat162float(mh)));
        ra[3 * D] = bf16_bits(one);
        ra[3 * D + 1] = bf16_bits(one);
        rb[3 * D] = bf16_bits(mh);
        rb[3 * D + 1] = bf16_bits(ml);
    }
    // 8 bf16 (16 bytes) per core-matrix row segment
    for (int kg = 0; kg < K / 8; ++kg) {
        uint4 va, vb;
        va.x = ra[8 * kg + 0] | ((uint32_t)ra[8 * kg + 1] << 16);
        va.y = ra[8 * kg + 2] | ((uint32_t)ra[8 * kg + 3] << 16);
        va.z = ra[8 * kg + 4] | ((uint32_t)ra[8 * kg + 5] << 16);
        va.w = ra[8 * kg + 6] | ((uint32_t)ra[8 * kg + 7] << 16);
        vb.x = rb[8 * kg + 0] | ((uint32_t)rb[8 * kg + 1] << 16);
        vb.y = rb[8 * kg + 2] | ((uint32_t)rb[8 * kg + 3] << 16);
        vb.z = rb[8 * kg + 4] | ((uint32_t)rb[8 * kg + 5] << 16);
        vb.w = rb[8 * kg + 6] | ((uint32_t)rb[8 * kg + 7] << 16);
        const int64_t off = cm_off(s, 8 * kg, K);
        *reinterpret_cast<uint4*>(tcA + off) = va;
        *reinterpret_cast<uint4*>(tcB + off) = vb;
    }
    tcn[s] = n;
    if (real) atomicMax(tcnu + e, float_to_ordered(n));
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
    unsigned long long* stat_survivors;   // pre-filter survivors (false-candidate rate)
    unsigned long long* stat_accepted;    // exact accepts
};

// Chunk geometry of a task: neighbour row L covers slot range [rs, re); its
// operand rows start at b8 = rs rounded down to 8 and end at e8 = re rounded
// up to 8; chunks of up to 256 rows (the MMA N, rounded up to 16).
struct ChunkTab {
    int rs[kTcMaxRows], re[kTcMaxRows], b8[kTcMaxRows], pref[kTcMaxRows + 1];
    int nrows, nch;
};

__device__ __forceinline__ void chunk_info(const ChunkTab& t, int c, int& start, int& n, int& lo,
                                           int& hi) {
    int L = 0;
    while (L + 1 < t.nrows && t.pref[L + 1] <= c) ++L;
    start = t.b8[L] + (c - t.pref[L]) * kTcN;
    const int e8 = (t.re[L] + 7) & ~7;
    n = min(kTcN, e8 - start);
    n = (n + 15) & ~15;
    lo = t.rs[L];
    hi = t.re[L];
}

template <int KS>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_query(TcArgs a) {
    constexpr int K = 16 * KS;
    constexpr int LCAP = tc_list_cap(KS);
    extern __shared__ __align__(1024) unsigned char smem[];
    const int D = a.D;
    const int DP = padded_dim(D);
    uint16_t* As = reinterpret_cast<uint16_t*>(smem);
    uint16_t* Bs = As + kTcM * K;
    float* Fs = reinterpret_cast<float*>(Bs + kTcRing * kTcN * K);
    float* Ld = Fs + kTcRing * kTcN * DP;
    int32_t* Li = reinterpret_cast<int32_t*>(Ld + LCAP * kTcLStr);

    __shared__ __align__(8) uint64_t bar_a, bar_b[kTcRing], bar_mma[2], bar_free[2];
    __shared__ uint32_t s_taddr;
    __shared__ Task s_task;
    __shared__ int s_done, s_abort;
    __shared__ ChunkTab s_ct;
    __shared__ int s_cnt[kTcThreads];
    __shared__ int s_lost[kTcThreads];
    __shared__ int s_qorig[kTcM];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int row = 32 * quarter + lane;   // TMEM lane / query row in the tile

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&s_taddr))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar_a, 1);
        for (int i = 0; i < kTcRing; ++i) mbar_init(&bar_b[i], 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_mma[i], 1);
            mbar_init(&bar_free[i], kTcThreads);
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
    int issued_loads = 0;     // producer bookkeeping (thread 0): chunks loaded / MMAs issued
    int issued_mma = 0;
    unsigned long long n_surv = 0, n_acc = 0;

    // producer helpers (thread 0 only)
    auto load_chunk = [&](int c, uint32_t g) {
        int start, n, lo, hi;
        chunk_info(s_ct, c, start, n, lo, hi);
        const int slot = g % kTcRing;
        const uint32_t bB = (uint32_t)n * K * 2;
        const uint32_t bF = (uint32_t)n * DP * 4;
        mbar_arrive_expect_tx(&bar_b[slot], bB + bF);
        bulk_g2s(Bs + (size_t)slot * kTcN * K, a.tcB + cm_off(start, 0, K), bB, &bar_b[slot]);
        bulk_g2s(Fs + (size_t)slot * kTcN * DP, a.rpts + (int64_t)(start >> 1) * 2 * DP, bF,
                 &bar_b[slot]);
    };
    auto abort_now = [&]() {
        atomicOr(a.status, kStatusTimeout);
        atomicExch(&s_abort, 1);
    };
    auto aborted = [&]() -> int { return *reinterpret_cast<volatile int*>(&s_abort); };
    auto issue_mma = [&](int c, uint32_t g) -> bool {
        const int slot = g % kTcRing;
        if (!mbar_wait_bounded(&bar_b[slot], (g / kTcRing) & 1u)) return false;
        if (g >= 2 && !mbar_wait_bounded(&bar_free[g & 1], ((g - 2) >> 1) & 1u)) return false;
        tc_fence_after();
        int start, n, lo, hi;
        chunk_info(s_ct, c, start, n, lo, hi);
        const uint32_t idesc = mma_idesc(n);
        const uint32_t bbase = sB + (uint32_t)(slot * kTcN * K * 2);
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            mma_bf16(taddr + (g & 1) * kTcN, smem_desc(sA + ks * 256, lbo, sbo),
                     smem_desc(bbase + ks * 256, lbo, sbo), idesc, ks > 0 ? 1u : 0u);
        }
        mma_commit(&bar_mma[g & 1]);
        return true;
    };

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const int t = atomicAdd(a.task_counter, 1);
            s_done = (t >= ntasks) || aborted();
            if (t < ntasks) s_task = a.tasks[t];
        }
        __syncthreads();
        if (s_done) break;
        const Task tk = s_task;
        const EventHdr& h = a.ev[tk.ev];
        int32_t* counts = a.counts ? a.counts : h.counts;
        int32_t* oidx = a.counts ? a.idx : h.idx;
        float* od2 = a.counts ? a.dist2 : h.dist2;
        const int w0 = tk.qslot & ~7;
        const int qs = w0 + row;
        const bool active = qs >= tk.qslot && qs < tk.qslot + tk.nq;
        const int qorig = active ? a.qperm[qs] : 0;
        if (half == 0) s_qorig[row] = qorig;
        if (!h.valid) {
            // grid built from non-finite input: empty rows (frnn_sync reports it)
            if (half == 0 && active) {
                for (int e = 0; e < Kout; ++e) {
                    oidx[(int64_t)qorig * Kout + e] = -1;
                    od2[(int64_t)qorig * Kout + e] = INFINITY;
                }
                counts[qorig] = 0;
            }
            continue;
        }
        // neighbour rows and chunk table (warp 0)
        if (warp == 0) {
            const int dims0 = h.dims[0], dims1 = h.dims[1], dims2 = h.dims[2], m = h.m;
            const int xa = a.qcell[tk.qslot] % dims0;
            const int xb = a.qcell[tk.qslot + tk.nq - 1] % dims0;
            const int y = tk.row % dims1, z = tk.row / dims1;
            const int side = 2 * m + 1;
            const int nrows = h.naxes >= 3 ? side * side : (h.naxes == 2 ? side : 1);
            int rs = 0, re = 0;
            if (lane < nrows) {
                const int dy = h.naxes >= 2 ? (lane % side) - m : 0;
                const int dz = h.naxes >= 3 ? (lane / side) - m : 0;
                const int yy = y + dy, zz = z + dz;
                if (yy >= 0 && yy < dims1 && zz >= 0 && zz < dims2) {
                    const int64_t rowbase = h.cell_off + (int64_t)(yy + dims1 * zz) * dims0;
                    rs = a.cstart[rowbase + max(xa - m, 0)];
                    re = a.cstart[rowbase + min(xb + m, dims0 - 1) + 1];
                }
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
            if (lane < kTcMaxRows) {
                s_ct.rs[lane] = rs;
                s_ct.re[lane] = re;
                s_ct.b8[lane] = b8;
                s_ct.pref[lane] = pre - nch;
            }
            if (lane == 31) {
                s_ct.nch = pre;
                s_ct.nrows = nrows;
            }
        }
        __syncthreads();
        const int nch = s_ct.nch;

        // this thread's query: float32 coordinates and the pass threshold
        float q[kMaxD];
#pragma unroll
        for (int k = 0; k < kMaxD; ++k)
            q[k] = (active && k < D) ? a.qpts[pair_index(qs, k, DP)] : 0.f;
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
        int cnt = 0;
        bool lost = false;

        if (nch > 0 && tid == 0) {
            // A tile + the first two chunks, then the first MMA
            const uint32_t bA = (uint32_t)kTcM * K * 2;
            mbar_arrive_expect_tx(&bar_a, bA);
            bulk_g2s(As, a.tcA + cm_off(w0, 0, K), bA, &bar_a);
            load_chunk(0, g0);
            if (nch > 1) load_chunk(1, g0 + 1);
            issued_loads = min(nch, 2);
            issued_mma = 0;
            if (!mbar_wait_bounded(&bar_a, task_no & 1u)) abort_now();
            else if (!issue_mma(0, g0)) abort_now();
            else issued_mma = 1;
        }
        for (int c = 0; c < nch; ++c) {
            const uint32_t g = g0 + c;
            if (tid == 0 && !aborted()) {
                if (c + 1 < nch) {
                    if (!issue_mma(c + 1, g + 1)) abort_now();
                    else issued_mma = c + 2;
                }
                // the epilogue of chunk c-1 is done (waited inside issue_mma),
                // so ring slot (c+2) % 3 is free again
                if (!aborted() && c + 2 < nch) {
                    load_chunk(c + 2, g + 2);
                    issued_loads = c + 3;
                }
            }
            // MMA done (accumulator ready) and the chunk's staged coordinates
            // visible to this thread
            if (!aborted()) {
                if (!mbar_wait_bounded(&bar_mma[g & 1], (g >> 1) & 1u) ||
                    !mbar_wait_bounded(&bar_b[g % kTcRing], (g / kTcRing) & 1u))
                    abort_now();
            }
            __syncwarp();
            tc_fence_after();
            if (!__shfl_sync(0xffffffffu, aborted(), 0)) {
                int start, n, lo, hi;
                chunk_info(s_ct, c, start, n, lo, hi);
                const float* F = Fs + (size_t)(g % kTcRing) * kTcN * DP;
                const uint32_t tbase = taddr + ((uint32_t)(32 * quarter) << 16) + (g & 1) * kTcN;
#pragma unroll 1
                for (int grp = 0; grp < 4; ++grp) {
                    const int col0 = half * 128 + grp * 32;
                    if (col0 >= n) break;                       // warp-uniform
                    float v[32];
                    __syncwarp();
                    tmem_ld32(tbase + col0, v);
                    const int nval = min(32, n - col0);
                    float mx = -INFINITY;
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const float v0 = j < nval ? v[j] : -INFINITY;
                        const float v1 = j + 1 < nval ? v[j + 1] : -INFINITY;
                        mx = fmax3(mx, v0, v1);
                    }
                    if (mx >= tx) {
                        uint32_t mask = 0;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < nval && v[j] >= tx) mask |= 1u << j;
                        while (mask) {
                            const int j = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const int cs = start + col0 + j;
                            if (cs < lo || cs >= hi || cs == self_slot) continue;
                            ++n_surv;
                            // exact contract from the staged float32 coordinates
                            const float* f = F + ((cs - start) >> 1) * 2 * DP + (cs & 1);
                            float sv = 0.f;
#pragma unroll
                            for (int k = 0; k < kMaxD; ++k) {
                                if (k < D) {
                                    const float d = __fsub_rn(q[k], f[2 * k]);
                                    sv = __fadd_rn(sv, __fmul_rn(d, d));
                                }
                            }
                            if (sv <= r2) {
                                ++n_acc;
                                if (cnt < LCAP) {
                                    Ld[cnt * kTcLStr + tid] = sv;
                                    Li[cnt * kTcLStr + tid] = a.rperm[cs];
                                } else {
                                    lost = true;
                                }
                                ++cnt;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&bar_free[g & 1]);
        }
        __syncthreads();
        if (aborted()) {
            // drain what thread 0 issued (bounded), then leave
            if (tid == 0) {
                for (int c = issued_mma; c < issued_loads; ++c)
                    mbar_wait_bounded(&bar_b[(g0 + c) % kTcRing], ((g0 + c) / kTcRing) & 1u);
                if (issued_mma > 0)
                    mbar_wait_bounded(&bar_mma[(g0 + issued_mma - 1) & 1],
                                      ((g0 + issued_mma - 1) >> 1) & 1u);
            }
            break;
        }
        g0 += nch;
        if (nch > 0) ++task_no;

        // merge the two column halves of each row, sort, count
        s_cnt[tid] = cnt;
        s_lost[tid] = lost ? 1 : 0;
        __syncthreads();
        if (half == 0 && active) {
            const int pt = tid + 128;
            int c1 = s_cnt[pt];
            bool l = lost || s_lost[pt] || cnt + c1 > LCAP;
            if (!l) {
                for (int e = 0; e < c1; ++e) {
                    Ld[(cnt + e) * kTcLStr + tid] = Ld[e * kTcLStr + pt];
                    Li[(cnt + e) * kTcLStr + tid] = Li[e * kTcLStr + pt];
                }
                cnt += c1;
                for (int e = 1; e < cnt; ++e) {
                    const float kd = Ld[e * kTcLStr + tid];
                    const int ki = Li[e * kTcLStr + tid];
                    int j = e - 1;
                    while (j >= 0) {
                        const float dj = Ld[j * kTcLStr + tid];
                        const int ij = Li[j * kTcLStr + tid];
                        if (dj < kd || (dj == kd && ij < ki)) break;
                        Ld[(j + 1) * kTcLStr + tid] = dj;
                        Li[(j + 1) * kTcLStr + tid] = ij;
                        --j;
                    }
                    Ld[(j + 1) * kTcLStr + tid] = kd;
                    Li[(j + 1) * kTcLStr + tid] = ki;
                }
                counts[qorig] = min(cnt, Kout);
                s_cnt[tid] = cnt;
                s_lost[tid] = 0;
            } else {
                s_lost[tid] = 1;
                const int pos = atomicAdd(a.ovf_count, 1);
                if (pos < a.ovf_cap) {
                    a.ovf[pos].qslot = qs;
                    a.ovf[pos].ev = tk.ev;
                } else {
                    atomicOr(a.status, kStatusCapacity);
                }
            }
        }
        if (half == 0 && !active) s_lost[tid] = 1;   // nothing to write for this row
        __syncthreads();
        // coalesced row writes: warp w writes rows 16w .. 16w + 15
        for (int rr = 0; rr < 16; ++rr) {
            const int r = warp * 16 + rr;
            if (s_lost[r]) continue;
            const int c = min(s_cnt[r], Kout);
            const int qo = s_qorig[r];
            int32_t* irow = oidx + (int64_t)qo * Kout;
            float* drow = od2 + (int64_t)qo * Kout;
            for (int e = lane; e < Kout; e += 32) {
                const bool real = e < c;
                irow[e] = real ? Li[e * kTcLStr + r] : -1;
                drow[e] = real ? Ld[e * kTcLStr + r] : INFINITY;
            }
        }
    }
    if (a.stat_survivors) {
        atomicAdd(a.stat_survivors, n_surv);
        atomicAdd(a.stat_accepted, n_acc);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr)
                     : "memory");
    }
}

// ------------------------------------------------------------- host

void tc_free(GridBufs& g) {
    if (g.tc_base) cudaFree(g.tc_base);
    g.tc_base = nullptr;
    g.tc_bytes = 0;
    g.tc_cap_rows = g.tc_cap_tasks = g.tc_cap_E = 0;
    g.tc_ready = false;
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Allocate (or keep) the operand buffers of a point set; enqueues nothing but
// the one-time zeroing of a fresh allocation (on the legacy default stream,
// synchronised, so it may run before a capture begins).
frnn_status tc_reserve(GridBufs& g, std::string& err) {
    const int K = tc_k_for(g.D);
    const int64_t rows = (g.n_total + 7) / 8 * 8 + kTcRowPad;
    int64_t tcap = 0;
    for (int e = 0; e < g.E; ++e)
        tcap += g.h_hdr[e].n / kTcM + g.h_hdr[e].cell_cap + 2;
    if (g.tc_base && g.tc_K == K && g.tc_cap_rows >= rows && g.tc_cap_tasks >= tcap &&
        g.tc_cap_E >= g.E)
        return FRNN_OK;
    tc_free(g);
    const size_t bA = al256(sizeof(uint16_t) * rows * K);
    const size_t bn = al256(sizeof(float) * rows);
    const size_t bnu = al256(sizeof(int32_t) * std::max(g.E, 1));
    const size_t bt = al256(sizeof(Task) * tcap);
    void* base = nullptr;
    cudaError_t ce = cudaMalloc(&base, 2 * bA + bn + bnu + bt + 256);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        err = "cudaMalloc of tensor-core operands failed";
        return FRNN_ERR_OUT_OF_MEMORY;
    }
    char* b = static_cast<char*>(base);
    g.tc_base = base;
    g.tc_bytes = 2 * bA + bn + bnu + bt + 256;
    g.tcA = reinterpret_cast<uint16_t*>(b);
    g.tcB = reinterpret_cast<uint16_t*>(b + bA);
    g.tcn = reinterpret_cast<float*>(b + 2 * bA);
    g.tcnu = reinterpret_cast<int32_t*>(b + 2 * bA + bn);
    g.tc_tasks = reinterpret_cast<Task*>(b + 2 * bA + bn + bnu);
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

frnn_status tc_prepare(GridBufs& g, const GridBufs& center_src, cudaStream_t st,
                       std::string& err) {
    frnn_status s0 = tc_reserve(g, err);
    if (s0 != FRNN_OK) return s0;
    const int K = tc_k_for(g.D);
    cudaMemsetAsync(g.tcnu, 0, sizeof(int32_t) * g.E, st);   // ordered(0.0f) == 0
    if (g.n_total > 0) {
        k_tc_prep<<<(unsigned)ceil_div(g.n_total, 128), 128, 0, st>>>(
            g.hdr, center_src.hdr, g.E, g.D, g.n_total, g.pts, g.tcA, g.tcB, g.tcn, g.tcnu, K);
    }
    enqueue_tasks(g, kTcM, 8, g.tc_tasks, g.scalars + kScTcTasks, st);
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
    const int KS = K / 16;
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
    a.stat_survivors = q.tc_stats;
    a.stat_accepted = q.tc_stats ? q.tc_stats + 1 : nullptr;
    cudaMemsetAsync(qs.scalars + kScOvfCount, 0, sizeof(int32_t), st);
    cudaMemsetAsync(qs.scalars + kScTcCounter, 0, sizeof(int32_t), st);
    const size_t smem = tc_smem_bytes(KS, padded_dim(D));
    cudaError_t ce = cudaSuccess;
    auto launch = [&](auto kern) {
        ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ce == cudaSuccess) {
            kern<<<q.num_sms, kTcThreads, smem, st>>>(a);
            ce = cudaGetLastError();
        }
    };
    if (KS == 2) launch(k_tc_query<2>);
    else if (KS == 3) launch(k_tc_query<3>);
    else if (KS == 4) launch(k_tc_query<4>);
    else {
        err = "tensor-core path: unsupported D";
        return FRNN_ERR_UNSUPPORTED;
    }
    if (ce != cudaSuccess) {
        err = std::string("tensor-core query launch failed: ") + cudaGetErrorString(ce);
        return FRNN_ERR_CUDA;
    }
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
    return enqueue_overflow(o, q.num_sms, st, err);
}

}  // namespace frnn
