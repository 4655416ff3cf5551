// match_tc.cu -- the brute-force Hamming matcher (Sec. III-B, ratio test of
// Sec. IV-C) on the 5th-generation tensor cores.
//
// A 256-bit descriptor becomes 256 fp8 (e4m3) values, +1 for a 0 bit and -1 for
// a 1 bit; then q.t = 256 - 2 H(q, t) exactly (every product is +-1 and an fp32
// sum of at most 256 of them is exact).  A CTA owns one SM and works through a
// contiguous range of items of (problem, 256 queries, train slice), numbered
// query-block-major: consecutive items of one query block (a run) share the
// query tile, loaded once, and the epilogue's running top two, so that its
// threshold is not reset at every slice boundary (slices folded into a run
// leave empty partial keys):
//   warp 0     TMA producer: the item's query tile (2 x 128 rows) once, then
//              128-row train tiles through a kTcStages-deep ring (K-major,
//              128-byte swizzle, two 128-byte column halves per tile),
//   warp 1     allocates the 512 TMEM columns and issues the MMAs (one thread):
//              per train tile, 2 query blocks x 8 tcgen05.mma (M = 128,
//              N = 128, K = 32) into accumulator stage s of 2,
//   warps 2-9  epilogue: thread = one TMEM lane = one query of one block; reads
//              128 columns with tcgen05.ld and keeps the nearest and
//              second-nearest as packed keys (distance << 23 | train index).
//              A 32-column chunk is inspected element by element only when its
//              largest dot product beats the current second best.
// The per-slice partial keys have the CUDA-core matcher's format, so its merge
// kernel finishes the job.  Every mbarrier wait is bounded by the global
// timer: on expiry the CTA records ASIFT_ERR_TIMEOUT, stops issuing, waits
// (bounded) for its own copies and MMAs in flight and frees its TMEM.
#include <atomic>

#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace asift {

constexpr int kTcBM = 128;                       // queries per MMA block (TMEM lanes)
constexpr int kTcQB = 2;                         // query blocks per item
constexpr int kTcBN = 128;                       // trains per tile (MMA N)
constexpr int kTcK = 256;                        // bytes per expanded descriptor
constexpr int kTcStages = 4;                     // train-tile ring depth
constexpr int kTcEpiWarps = 4 * kTcQB;
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr int kTcAHalf = kTcQB * kTcBM * 128;    // one 128-byte column half of the query tile
constexpr int kTcBHalf = kTcBN * 128;
constexpr int kTcABytes = 2 * kTcAHalf;
constexpr int kTcBBytes = 2 * kTcBHalf;
constexpr int kTcSmem = kTcABytes + kTcStages * kTcBBytes + 256 + 1024;
constexpr int kTcCols = 2 * kTcQB * kTcBN;       // TMEM columns: 2 accumulator stages
constexpr unsigned kTcNoKey = 0xffffffffu;
constexpr int kMaxTcProblems = 512;

static_assert(kTcCols == 512, "the accumulators fill TMEM");
static_assert(kTcSmem <= 227 * 1024 - 8 * 1024, "shared memory budget");

// ---------------------------------------------------------------- PTX helpers
// Shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle: start address (16-byte units, bits 0-13), leading byte offset
// (unused by this layout, 1), stride byte offset 1024 (8-row groups, bits
// 32-45), descriptor version 1 (bit 46), swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: D fp32 (bits 4-5 = 1), A and B e4m3 (bits 7-9, 10-12
// = 0), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTcBN >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);

__device__ __forceinline__ void umma_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive fp32 columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- expansion
// Packed descriptor bytes (bit i of a row in byte i>>3 at position i&7) ->
// e4m3 +1 (0x38) for a 0 bit, -1 (0xB8) for a 1 bit; 8 output bytes per input.
__device__ __forceinline__ uint2 expand_byte(unsigned b)
{
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        lo |= (((b >> k) & 1u) ? 0xB8u : 0x38u) << (8 * k);
        hi |= (((b >> (k + 4)) & 1u) ? 0xB8u : 0x38u) << (8 * k);
    }
    return make_uint2(lo, hi);
}

// Group g (blockIdx.y) owns rows [first_view[g] * n_per_view, + count[g]) of
// the packed pool; only those rows are expanded.  d_first == NULL: one group
// of rows [0, count ? *count : cap).
__global__ void expand_pm1_kernel(const uint8_t *__restrict__ packed, uint8_t *__restrict__ out,
                                  const int32_t *__restrict__ d_first, int n_per_view,
                                  const int32_t *__restrict__ d_count, long long cap)
{
    const int g = blockIdx.y;
    const long long row0 = d_first ? (long long)d_first[g] * n_per_view : 0;
    long long rows = d_count ? (long long)max(d_count[g], 0) : cap;
    if (d_first) rows = min(rows, (long long)(d_first[g + 1] - d_first[g]) * n_per_view);
    else rows = min(rows, cap);
    const long long n = rows * 32;
    const uint8_t *src = packed + row0 * 32;
    uint2 *dst = reinterpret_cast<uint2 *>(out + row0 * 256);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = expand_byte(src[i]);
}

// ---------------------------------------------------------------- epilogue
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float max32(const float v[32])
{
    float m[11];
#pragma unroll
    for (int i = 0; i < 10; ++i) m[i] = max3f(v[3 * i], v[3 * i + 1], v[3 * i + 2]);
    m[10] = fmaxf(v[30], v[31]);
    const float a = max3f(m[0], m[1], m[2]), b = max3f(m[3], m[4], m[5]), c = max3f(m[6], m[7], m[8]);
    return max3f(max3f(a, b, c), m[9], m[10]);
}

// Inserts the key of the score s = 64 v - j (v the dot product, j the column
// in the chunk) into the running top two.  A key that is not below b2 leaves
// both unchanged, so candidates need no pre-test.
__device__ __forceinline__ void insert_score(float s, int col0, unsigned &b1, unsigned &b2)
{
    const int si = __float2int_rn(s);
    const int v = (si + 63) >> 6;                         // ceil(s / 64): the dot product
    const int j = (v << 6) - si;
    const unsigned key = ((unsigned)((256 - v) >> 1) << 23) | (unsigned)(col0 + j);
    b2 = min(b2, max(b1, key));
    b1 = min(b1, key);
}

// One 32-column chunk of a thread's accumulator row (dot products, even
// integers in [-256, 256]).  Only the chunk's two smallest keys (largest dot,
// then lowest column) can enter the top two, and none can unless the chunk's
// maximum beats the current second best (thr, its dot product): the common
// case costs 16 three-input max and one compare.  Columns only grow along a
// run, so the chunk's best key k1 is below b1 iff its dot beats b1's (best,
// its dot product); otherwise k1 becomes at most the new b2 and the chunk's
// second key, above k1, cannot enter, so the second pass runs only when the
// chunk beats the best.  kFull = false masks columns >= valid.
template <bool kFull>
__device__ __forceinline__ void epi_chunk(const uint32_t r[32], int valid, int col0, unsigned &b1, unsigned &b2,
                                          float &thr, float &best)
{
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = (kFull || j < valid) ? __uint_as_float(r[j]) : -1.0e30f;
    const float mx = max32(v);
    if (mx > thr) {
        float sc[32];                                     // 64 v - j: max gives the largest v, then lowest j
#pragma unroll
        for (int j = 0; j < 32; ++j) sc[j] = fmaf(v[j], 64.0f, -(float)j);
        const float s1 = max32(sc);
        if (mx > best) {
#pragma unroll
            for (int j = 0; j < 32; ++j) sc[j] = (sc[j] == s1) ? -3.0e30f : sc[j];
            const float s2 = max32(sc);
            insert_score(s1, col0, b1, b2);
            if (s2 > -1.0e20f) insert_score(s2, col0, b1, b2);
        } else {
            insert_score(s1, col0, b1, b2);
        }
        thr = (b2 == kTcNoKey) ? -1.0e30f : 256.0f - 2.0f * (float)(b2 >> 23);
        best = (b1 == kTcNoKey) ? -1.0e30f : 256.0f - 2.0f * (float)(b1 >> 23);
    }
}

// ---------------------------------------------------------------- the matcher
__device__ __forceinline__ int tc_count(const int32_t *d, int cap) { return d ? min(max(*d, 0), cap) : cap; }

struct TcItem {
    int p, split, qblk, t0, t1;
};

__device__ __forceinline__ bool same_run(const TcItem &a, const TcItem &b) { return a.p == b.p && a.qblk == b.qblk; }

__global__ void __launch_bounds__(kTcThreads, 1)
hamming_tc_kernel(const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap tmap,
                  const uint4 *qbase, const uint4 *tbase, const MatchProblem *__restrict__ many, int n_probs,
                  const MatchProblem single, int target_items, int32_t *status, unsigned long long stall_ns)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *smA = base;                                     // [2 halves][2 blocks x 128 rows][128 B]
    uint8_t *smB = base + kTcABytes;                         // [stage][2 halves][128 rows][128 B]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smB + kTcStages * kTcBBytes);
    uint64_t *full = bars, *empty = bars + kTcStages;
    uint64_t *acc_full = bars + 2 * kTcStages, *acc_empty = acc_full + 2;
    uint64_t *a_full = acc_empty + 2, *a_empty = a_full + 1;
    uint64_t *never = a_empty + 1;                           // failure-path test: nothing arrives here
    const unsigned long long lim = stall_ns ? stall_ns : kTmaWaitNs;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_sh;
    __shared__ int s_items[kMaxTcProblems + 1], s_chunk[kMaxTcProblems], s_nsplit[kMaxTcProblems];
    volatile int *abort_flag = &abort_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = many ? n_probs : 1;
    if (threadIdx.x == 0) {
        abort_sh = 0;
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], kTcEpiWarps);
        }
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // Slicing: about target_items items over all problems, in proportion
        // to each problem's nq x nt; chunks are whole train tiles.
        double total = 0.0;
        for (int p = 0; p < np; ++p) {
            const MatchProblem &P = many ? many[p] : single;
            total += (double)tc_count(P.d_nq, P.nq_cap) * (double)tc_count(P.d_nt, P.nt_cap);
        }
        int acc = 0;
        for (int p = 0; p < np; ++p) {
            const MatchProblem &P = many ? many[p] : single;
            const int nq = tc_count(P.d_nq, P.nq_cap), nt = tc_count(P.d_nt, P.nt_cap);
            const int qb = (nq + kTcQB * kTcBM - 1) / (kTcQB * kTcBM);
            int ns = 0, ch = kTcBN;
            if (nq > 0 && nt > 0) {
                const double w = (double)nq * (double)nt / total;
                int s = max(1, ((int)(target_items * w) + qb - 1) / qb);
                s = min(s, (nt + kTcBN - 1) / kTcBN);
                s = max(1, min(s, P.s_alloc));
                ch = ((nt + s - 1) / s + kTcBN - 1) / kTcBN * kTcBN;
                ns = (nt + ch - 1) / ch;
            }
            s_chunk[p] = ch;
            s_nsplit[p] = ns;
            s_items[p] = acc;
            acc += ns * qb;
            if (blockIdx.x == 0) {
                P.plan[0] = ns;
                P.plan[1] = ch;
            }
        }
        s_items[np] = acc;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int items = s_items[np];
    // this CTA's items: a contiguous range (equal shares, one item apart at most)
    const int i_lo = (int)((long long)items * blockIdx.x / gridDim.x);
    const int i_hi = (int)((long long)items * (blockIdx.x + 1) / gridDim.x);

    // items are visited in increasing order, so the owning problem only moves
    // forward; within a problem item = query block * slices + slice
    auto item_of = [&](int item, int &p) {
        while (s_items[p + 1] <= item) ++p;
        const MatchProblem &P = many ? many[p] : single;
        const int nt = tc_count(P.d_nt, P.nt_cap);
        const int local = item - s_items[p], ns = s_nsplit[p];
        TcItem it;
        it.p = p;
        it.qblk = local / ns;
        it.split = local - it.qblk * ns;
        it.t0 = it.split * s_chunk[p];
        it.t1 = min(nt, it.t0 + s_chunk[p]);
        return it;
    };
    // whether item (> i_lo) continues the run of item - 1, and whether item
    // (< i_hi - 1) is followed by one of its run
    auto continues = [&](int item, int p) {
        if (item <= i_lo) return false;
        int q = p;
        const TcItem a = item_of(item - 1, q), b = item_of(item, q);
        return same_run(a, b);
    };

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int stage = 0, p = 0;
            uint32_t ph = 0, a_ph = 0;
            unsigned used = 0, par = 0;        // stages with a load issued, parity of their last load
            bool a_used = false;
            for (int item = i_lo; item < i_hi && !*abort_flag; ++item) {
                const bool cont = continues(item, p);
                const TcItem it = item_of(item, p);
                const MatchProblem &P = many ? many[it.p] : single;
                const int qrow = (int)((P.q - qbase) >> 1) + it.qblk * kTcQB * kTcBM;
                const int trow = (int)((P.t - tbase) >> 1);
                if (!cont) {   // a new run: its query tile, once the previous run's MMAs are done with smA
                    if (!mbar_wait(a_empty, a_ph ^ 1, abort_flag, status, lim)) break;
                    mbar_expect_tx(a_full, kTcABytes);
                    tma_load_2d(smA, &qmap, 0, qrow, a_full);
                    tma_load_2d(smA + kTcAHalf, &qmap, 128, qrow, a_full);
                    a_used = true;
                    a_ph ^= 1;
                }
                bool ok = true;
                for (int tb = it.t0; tb < it.t1; tb += kTcBN) {
                    if (!mbar_wait(&empty[stage], ph ^ 1, abort_flag, status, lim)) { ok = false; break; }
                    uint8_t *dst = smB + stage * kTcBBytes;
                    mbar_expect_tx(&full[stage], kTcBBytes);
                    tma_load_2d(dst, &tmap, 0, trow + tb, &full[stage]);
                    tma_load_2d(dst + kTcBHalf, &tmap, 128, trow + tb, &full[stage]);
                    used |= 1u << stage;
                    par = (par & ~(1u << stage)) | (ph << stage);
                    if (++stage == kTcStages) { stage = 0; ph ^= 1; }
                }
                if (!ok) break;
            }
            // own copies in flight complete before the CTA can leave
            for (int s = 0; s < kTcStages; ++s)
                if (used >> s & 1u) mbar_wait(&full[s], (par >> s) & 1u, nullptr, status);
            if (a_used) mbar_wait(a_full, a_ph ^ 1, nullptr, status);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int stage = 0, acc = 0, p = 0, last_acc = -1;
            uint32_t ph = 0, acc_ph = 0, a_ph = 0, last_par = 0;
            const uint32_t a0 = smem_u32(smA), b0 = smem_u32(smB);
            // failure-path test: a wait that runs out (no copy or MMA depends
            // on `never`); it raises the abort flag, which every role sees
            if (stall_ns) mbar_wait(never, 0, abort_flag, status, lim);
            for (int item = i_lo; item < i_hi && !*abort_flag; ++item) {
                const bool cont = continues(item, p);
                const bool last_of_run = item + 1 >= i_hi || !continues(item + 1, p);
                const TcItem it = item_of(item, p);
                if (!cont) {
                    if (!mbar_wait(a_full, a_ph, abort_flag, status, lim)) break;
                    a_ph ^= 1;
                }
                tc_fence_after();
                bool ok = true;
                for (int tb = it.t0; tb < it.t1; tb += kTcBN) {
                    if (!mbar_wait(&full[stage], ph, abort_flag, status, lim)) { ok = false; break; }
                    if (!mbar_wait(&acc_empty[acc], acc_ph ^ 1, abort_flag, status, lim)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t bs = b0 + (uint32_t)(stage * kTcBBytes);
#pragma unroll
                    for (int qb = 0; qb < kTcQB; ++qb) {
                        const uint32_t d = tmem + (uint32_t)((acc * kTcQB + qb) * kTcBN);
#pragma unroll
                        for (int k = 0; k < kTcK / 32; ++k) {
                            // k-th 32-byte step: column half k/4, offset (k%4)*32 inside the swizzle row
                            const uint32_t koff = (uint32_t)((k & 3) * 32);
                            const uint64_t ad =
                                umma_desc(a0 + (uint32_t)((k >> 2) * kTcAHalf + qb * kTcBM * 128) + koff);
                            const uint64_t bd = umma_desc(bs + (uint32_t)((k >> 2) * kTcBHalf) + koff);
                            umma_f8(d, ad, bd, k > 0 ? 1u : 0u);
                        }
                    }
                    umma_commit(&empty[stage]);
                    umma_commit(&acc_full[acc]);
                    last_acc = acc;
                    last_par = acc_ph;
                    if (++stage == kTcStages) { stage = 0; ph ^= 1; }
                    if (++acc == 2) { acc = 0; acc_ph ^= 1; }
                }
                if (last_of_run || !ok) umma_commit(a_empty);   // the run's MMAs release smA
                if (!ok) break;
            }
            // the MMAs issued have finished before TMEM is freed
            if (last_acc >= 0) mbar_wait(&acc_full[last_acc], last_par, nullptr, status);
        }
    } else {
        // ---------------- epilogue: one TMEM lane (= one query) per thread
        const int quarter = warp & 3;                    // TMEM lanes this warp may access
        const int qb = (warp - 2) >> 2;                  // query block of this warp
        const int row = qb * kTcBM + quarter * 32 + lane;
        int acc = 0, p = 0;
        uint32_t acc_ph = 0;
        unsigned b1 = kTcNoKey, b2 = kTcNoKey;
        float thr = -1.0e30f, best = -1.0e30f;           // dot products of b2 and b1 (-inf: none)
        for (int item = i_lo; item < i_hi && !*abort_flag; ++item) {
            const bool cont = continues(item, p);
            const bool last_of_run = item + 1 >= i_hi || !continues(item + 1, p);
            const TcItem it = item_of(item, p);
            const MatchProblem &P = many ? many[it.p] : single;
            const int nq = tc_count(P.d_nq, P.nq_cap);
            if (!cont) {
                b1 = b2 = kTcNoKey;
                thr = best = -1.0e30f;
            }
            bool ok = true;
            for (int tb = it.t0; tb < it.t1; tb += kTcBN) {
                if (!mbar_wait(&acc_full[acc], acc_ph, abort_flag, status, lim)) { ok = false; break; }
                tc_fence_after();
                const uint32_t taddr =
                    tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((acc * kTcQB + qb) * kTcBN);
                const int valid = min(kTcBN, it.t1 - tb);
                __syncwarp();                            // tcgen05.ld is warp-collective
                uint32_t r[kTcBN / 32][32];              // the whole tile row: one wait per tile
#pragma unroll
                for (int c = 0; c < kTcBN / 32; ++c) tmem_ld32(taddr + (uint32_t)(c * 32), r[c]);
                tmem_wait_ld();
                if (valid == kTcBN) {
#pragma unroll
                    for (int c = 0; c < kTcBN / 32; ++c) epi_chunk<true>(r[c], 32, tb + c * 32, b1, b2, thr, best);
                } else {
#pragma unroll
                    for (int c = 0; c < kTcBN / 32; ++c)
                        epi_chunk<false>(r[c], valid - c * 32, tb + c * 32, b1, b2, thr, best);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[acc]);
                if (++acc == 2) { acc = 0; acc_ph ^= 1; }
            }
            if (!ok) break;
            // a run's top two go to its last slice; the slices folded into it get none
            const int qi = it.qblk * kTcQB * kTcBM + row;
            if (qi < nq)
                P.part[(size_t)it.split * P.nq_cap + qi] = last_of_run ? make_uint2(b1, b2) : make_uint2(kTcNoKey, kTcNoKey);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
    }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// 2-D map over `rows` expanded descriptors (256 bytes each): box 128 bytes x
// box_rows, 128-byte swizzle, rows past the end read as zeros.
static cudaError_t make_map(CUtensorMap *m, const void *ptr, long long rows, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if (!ptr || (reinterpret_cast<uintptr_t>(ptr) & 15) || rows <= 0 || rows > INT32_MAX) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)kTcK, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kTcK};
    const cuuint32_t box[2] = {128, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Compute capability 10.x and the tensor-map encoder present (cached per device).
bool tc_match_available()
{
    static std::atomic<int> cache[64] = {};   // 0 unknown, 1 no, 2 yes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c) return c == 2;
    }
    int major = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
    const bool ok = major == 10 && encode_fn() != nullptr;
    if (dev >= 0 && dev < 64) cache[dev].store(ok ? 2 : 1, std::memory_order_relaxed);
    return ok;
}

size_t tc_expanded_bytes(long long rows) { return (size_t)std::max<long long>(rows, 1) * kTcK; }

cudaError_t launch_expand(const uint8_t *packed, uint8_t *out, const int32_t *d_first, int n_per_view,
                          const int32_t *d_count, long long cap_rows, int n_groups, cudaStream_t s)
{
    if (cap_rows <= 0 || n_groups <= 0) return cudaSuccess;
    const long long per_group = cap_rows * 32 / n_groups;
    const int bx = (int)std::max<long long>(1, std::min<long long>((per_group + 255) / 256, 8LL * device_sm_count() / n_groups + 1));
    expand_pm1_kernel<<<dim3(bx, n_groups), 256, 0, s>>>(packed, out, d_first, n_per_view, d_count, cap_rows);
    note_launch();
    return cudaGetLastError();
}

// Tensor-core matcher over problems whose query / train descriptors lie in
// the packed buffers starting at qbase / tbase; qexp / texp mirror them row
// for row in expanded form (q_rows / t_rows rows).  Then the shared merge.
cudaError_t launch_match_tc(const uint8_t *qbase, const uint8_t *qexp, long long q_rows, const uint8_t *tbase,
                            const uint8_t *texp, long long t_rows, const MatchProblem *d_probs, int n_probs,
                            const MatchProblem &single, int total_q, int num, int den, const MatchTuning &tune,
                            int32_t *status, cudaStream_t s)
{
    if (total_q <= 0) return cudaSuccess;
    if (n_probs > kMaxTcProblems) return cudaErrorInvalidValue;
    CUtensorMap qm, tm;
    cudaError_t e = make_map(&qm, qexp, q_rows, kTcQB * kTcBM);
    if (e == cudaSuccess) e = make_map(&tm, texp, t_rows, kTcBN);
    if (e != cudaSuccess) return e;
    e = ensure_dynamic_smem((const void *)hamming_tc_kernel, kTcSmem);
    if (e != cudaSuccess) return e;
    const int sms = device_sm_count();
    const int grid = tune.grid > 0 ? std::min(tune.grid, sms) : sms;   // one CTA per SM: it holds all of TMEM
    // about twelve items per CTA by default: the shorter runs cost more scalar
    // passes but balance the CTAs' ranges better (4 per CTA: 0.245 ms, 12: 0.233
    // ms for the matching stage of a 1024x768 pair)
    const int target = tune.target_items > 0 ? tune.target_items : 12 * grid;
    hamming_tc_kernel<<<grid, kTcThreads, kTcSmem, s>>>(qm, tm, reinterpret_cast<const uint4 *>(qbase),
                                                        reinterpret_cast<const uint4 *>(tbase), d_probs, n_probs,
                                                        single, target, status, tune.stall_ns);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_merge(d_probs, n_probs, single, total_q, num, den, s);
}

}  // namespace asift
