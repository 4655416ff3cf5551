// match.cu -- brute-force Hamming matching with the ratio test (Sec. III-B,
// Sec. IV-C) on sm_103a, and the accepted-pair output of match_pair.
//
// One launch serves a list of independent problems (one per image pair):
// hamming_top2_kernel is persistent over (problem, train slice, query block)
// items.  Each thread keeps kMQ query descriptors (2 x uint4 each) in
// registers; the CTA stages kMTile train descriptors in shared memory and every
// thread scans them.  The running nearest and second-nearest are kept as
// packed keys (distance << 23 | train index), so a min/max network gives the
// lowest index on distance ties and d2 counts equal distances.  merge_kernel
// takes the two smallest keys over a problem's slices (exact: keys are unique).
// How a problem is sliced is decided on the device from its actual pool sizes.
// The coarse stage's per-view match counts and their argmax live here too.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace asift {

constexpr int kMQ = 4;
constexpr int kMThreads = 128;
constexpr int kMTile = 256;
constexpr unsigned kNoKey = 0xffffffffu;
constexpr int kMaxMatchProblems = 512;

// Hamming distance of two 256-bit descriptors.  The eight XOR words are summed
// bit-sliced with carry-save adders (three-input XOR and majority, one LOP3
// each), leaving four words of weight 1, 2, 4 and 8: four popc instead of
// eight.
__device__ __forceinline__ void csa(unsigned a, unsigned b, unsigned c, unsigned &sum, unsigned &carry)
{
    sum = a ^ b ^ c;
    carry = (a & b) | (c & (a ^ b));
}

__device__ __forceinline__ unsigned ham256(const uint4 &a0, const uint4 &a1, const uint4 &b0, const uint4 &b1)
{
    const unsigned x0 = a0.x ^ b0.x, x1 = a0.y ^ b0.y, x2 = a0.z ^ b0.z, x3 = a0.w ^ b0.w;
    const unsigned x4 = a1.x ^ b1.x, x5 = a1.y ^ b1.y, x6 = a1.z ^ b1.z, x7 = a1.w ^ b1.w;
    unsigned s1, c1, s2, c2, s3, c3, t1, d1;
    csa(x0, x1, x2, s1, c1);
    csa(x3, x4, x5, s2, c2);
    csa(s1, s2, x6, s3, c3);
    const unsigned ones = s3 ^ x7, c4 = s3 & x7;          // weight 1; c1..c4 weight 2
    csa(c1, c2, c3, t1, d1);
    const unsigned twos = t1 ^ c4, d2 = t1 & c4;          // weight 2; d1, d2 weight 4
    const unsigned fours = d1 ^ d2, eights = d1 & d2;     // weight 4, 8
    return __popc(ones) + 2 * __popc(twos) + 4 * __popc(fours) + 8 * __popc(eights);
}

__device__ __forceinline__ const MatchProblem &prob(const MatchProblem *many, const MatchProblem &single, int i)
{
    return many ? many[i] : single;
}

__device__ __forceinline__ int count_of(const int32_t *d, int cap) { return d ? min(max(*d, 0), cap) : cap; }

// Slicing of one problem: about `target` items of kMThreads*kMQ queries x
// chunk trains, chunk a multiple of kMTile, at most s_alloc slices.
__device__ __forceinline__ void match_plan(int nq, int nt, int s_alloc, int target, int &n_split, int &chunk)
{
    n_split = 0;
    chunk = kMTile;
    if (nq <= 0 || nt <= 0) return;
    const int qblocks = (nq + kMThreads * kMQ - 1) / (kMThreads * kMQ);
    int s = max(1, (target + qblocks - 1) / qblocks);
    s = min(s, (nt + kMTile - 1) / kMTile);
    s = max(1, min(s, s_alloc));
    int c = (nt + s - 1) / s;
    c = ((c + kMTile - 1) / kMTile) * kMTile;
    chunk = c;
    n_split = (nt + c - 1) / c;
}

__global__ void __launch_bounds__(kMThreads, 7)
hamming_top2_kernel(const MatchProblem *__restrict__ many, int n_probs, const MatchProblem single, int target_items)
{
    __shared__ uint4 st[2 * kMTile];
    __shared__ int s_items[kMaxMatchProblems + 1];      // item prefix over problems
    __shared__ int s_chunk[kMaxMatchProblems], s_qblocks[kMaxMatchProblems];
    const int np = many ? n_probs : 1;
    if (threadIdx.x == 0) {
        // the target is shared out in proportion to each problem's pair count
        double total = 0.0;
        for (int p = 0; p < np; ++p) {
            const MatchProblem &P = prob(many, single, p);
            total += (double)count_of(P.d_nq, P.nq_cap) * (double)count_of(P.d_nt, P.nt_cap);
        }
        int acc = 0;
        for (int p = 0; p < np; ++p) {
            const MatchProblem &P = prob(many, single, p);
            const int nq = count_of(P.d_nq, P.nq_cap), nt = count_of(P.d_nt, P.nt_cap);
            const double w = total > 0 ? (double)nq * (double)nt / total : 0.0;
            const int tgt = max(1, (int)(target_items * w));
            int ns, ch;
            match_plan(nq, nt, P.s_alloc, tgt, ns, ch);
            s_chunk[p] = ch;
            s_qblocks[p] = (nq + kMThreads * kMQ - 1) / (kMThreads * kMQ);
            s_items[p] = acc;
            acc += ns * s_qblocks[p];
            if (blockIdx.x == 0) {
                P.plan[0] = ns;
                P.plan[1] = ch;
            }
        }
        s_items[np] = acc;
    }
    __syncthreads();
    const int items = s_items[np];
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        int p = 0;
        while (s_items[p + 1] <= item) ++p;
        const MatchProblem &P = prob(many, single, p);
        const int nq = count_of(P.d_nq, P.nq_cap), nt = count_of(P.d_nt, P.nt_cap);
        const int nq_cap = P.nq_cap;
        uint2 *__restrict__ part = P.part;
        const int local = item - s_items[p];
        const int qblocks = s_qblocks[p];
        const int split = local / qblocks, qb = local - split * qblocks;
        const int qbase = qb * (kMThreads * kMQ);
        const int t0 = split * s_chunk[p], t1 = min(nt, t0 + s_chunk[p]);
        const uint4 *__restrict__ q = P.q;
        const uint4 *__restrict__ t = P.t;
        uint4 qa[kMQ], qc[kMQ];
        unsigned b1[kMQ], b2[kMQ];
#pragma unroll
        for (int k = 0; k < kMQ; ++k) {
            const int qi = qbase + k * kMThreads + threadIdx.x;
            if (qi < nq) {
                qa[k] = q[2LL * qi];
                qc[k] = q[2LL * qi + 1];
            } else {
                qa[k] = make_uint4(0, 0, 0, 0);
                qc[k] = qa[k];
            }
            b1[k] = kNoKey;
            b2[k] = kNoKey;
        }
        for (int tb = t0; tb < t1; tb += kMTile) {
            const int nb = min(kMTile, t1 - tb);
            __syncthreads();
            for (int i = threadIdx.x; i < 2 * nb; i += blockDim.x) st[i] = t[2LL * tb + i];
            __syncthreads();
            for (int j = 0; j < nb; ++j) {
                const uint4 x0 = st[2 * j], x1 = st[2 * j + 1];
                const unsigned idx = (unsigned)(tb + j);
#pragma unroll
                for (int k = 0; k < kMQ; ++k) {
                    const unsigned key = (ham256(qa[k], qc[k], x0, x1) << 23) | idx;
                    b2[k] = min(b2[k], max(b1[k], key));
                    b1[k] = min(b1[k], key);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kMQ; ++k) {
            const int qi = qbase + k * kMThreads + threadIdx.x;
            if (qi < nq) part[(size_t)split * nq_cap + qi] = make_uint2(b1[k], b2[k]);
        }
    }
}

// One thread per query of every problem (problems laid end to end by q_off).
__global__ void __launch_bounds__(256)
merge_kernel(const MatchProblem *__restrict__ many, int n_probs, const MatchProblem single, int total_q, int num,
             int den)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    int p = 0;
    if (many) {
        int lo = 0, hi = n_probs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (many[mid].q_off <= g) lo = mid; else hi = mid - 1;
        }
        p = lo;
    }
    const MatchProblem &P = prob(many, single, p);
    const int qi = g - P.q_off;
    const int nq = count_of(P.d_nq, P.nq_cap), nt = count_of(P.d_nt, P.nt_cap);
    const int n_split = nt > 0 ? P.plan[0] : 0;
    bool acc = false;
    if (g < total_q && qi < nq) {
        unsigned b1 = kNoKey, b2 = kNoKey;
        for (int s = 0; s < n_split; ++s) {
            const uint2 pp = P.part[(size_t)s * P.nq_cap + qi];
            b2 = min(b2, max(b1, pp.x));
            b1 = min(b1, pp.x);
            b2 = min(b2, max(b1, pp.y));
            b1 = min(b1, pp.y);
        }
        asift_match m;
        m.best = (b1 == kNoKey) ? -1 : (int)(b1 & 0x7fffffu);
        m.d1 = (uint16_t)((b1 == kNoKey) ? 257 : (b1 >> 23));
        m.d2 = (uint16_t)((b2 == kNoKey) ? 257 : (b2 >> 23));
        acc = nt >= 2 && den * (int)m.d1 < num * (int)m.d2;
        P.out[qi] = m;
        if (P.accept) P.accept[qi] = (uint8_t)acc;
    }
    // one atomic per warp and problem (a warp can straddle two problems)
    const unsigned same = __match_any_sync(0xffffffffu, p);
    const unsigned bal = __ballot_sync(0xffffffffu, acc) & same;
    const int leader = __ffs(same) - 1;
    if ((int)(threadIdx.x & 31u) == leader && bal && P.n_acc) atomicAdd(P.n_acc, __popc(bal));
}

// ---------------------------------------------------------------- accepted pairs
constexpr int kPairBlock = 1024;

__device__ __forceinline__ int pair_problem(const MatchProblem *many, int n_probs, int block)
{
    if (!many) return 0;
    int lo = 0, hi = n_probs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (many[mid].blk_off <= block) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kPairBlock)
pair_count_kernel(const MatchProblem *__restrict__ many, int n_probs, const MatchProblem single,
                  int32_t *__restrict__ block_count)
{
    __shared__ int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int p = pair_problem(many, n_probs, blockIdx.x);
    const MatchProblem &P = prob(many, single, p);
    const int nq = count_of(P.d_nq, P.nq_cap);
    const int i = (blockIdx.x - P.blk_off) * kPairBlock + threadIdx.x;
    const bool a = i < nq && P.accept[i];
    const unsigned bal = __ballot_sync(0xffffffffu, a);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&s, __popc(bal));
    __syncthreads();
    if (threadIdx.x == 0) block_count[blockIdx.x] = s;
}

// Keypoint at (x, y) of level entry L -> source image pixel (the level's
// back-projection map, composed on the host in fp64).
__device__ __forceinline__ void backproject(const DevLevel &L, int x, int y, float *sx, float *sy)
{
    const double X = (double)x, Y = (double)y;
    *sx = (float)fma(L.bp[0], X, fma(L.bp[1], Y, L.bp[2]));
    *sy = (float)fma(L.bp[3], X, fma(L.bp[4], Y, L.bp[5]));
}

__global__ void __launch_bounds__(kPairBlock)
pair_write_kernel(const MatchProblem *__restrict__ many, int n_probs, const MatchProblem single,
                  const int32_t *__restrict__ block_count, const DevLevel *__restrict__ lv, int nv,
                  int32_t *__restrict__ status)
{
    __shared__ int wsum[kPairBlock / 32];
    __shared__ int base;
    const int p = pair_problem(many, n_probs, blockIdx.x);
    const MatchProblem &P = prob(many, single, p);
    const int lb = blockIdx.x - P.blk_off;
    const int nq = count_of(P.d_nq, P.nq_cap);
    if (threadIdx.x < 32) {   // this block's offset: the earlier blocks' counts, summed by warp 0
        int b = 0;
        for (int k = P.blk_off + (int)threadIdx.x; k < (int)blockIdx.x; k += 32) b += block_count[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (threadIdx.x == 0) base = b;
    }
    const int i = lb * kPairBlock + threadIdx.x;
    const bool a = i < nq && P.accept[i];
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, a);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < kPairBlock / 32; ++k) { const int v = wsum[k]; wsum[k] = acc; acc += v; }
        if (lb == P.n_blk - 1) {
            *P.d_n = base + acc;
            if (base + acc > P.cap) set_status(status, ASIFT_ERR_CAPACITY);
        }
    }
    __syncthreads();
    if (a) {
        const int o = base + wsum[w] + __popc(bal & ((1u << lane) - 1u));
        const asift_match mm = P.out[i];
        // a train index outside the pool can only come from a matcher launch
        // that gave up (status word set): such a pair is counted, not written
        if (o < P.cap && mm.best >= 0 && mm.best < count_of(P.d_nt, P.nt_cap)) {
            const asift_keypoint k1 = P.kp1[i], k2 = P.kp2[mm.best];
            asift_pair_match pm;
            backproject(lv[(size_t)k1.level * nv + k1.view], k1.x, k1.y, &pm.x1, &pm.y1);
            backproject(lv[(size_t)k2.level * nv + k2.view], k2.x, k2.y, &pm.x2, &pm.y2);
            pm.q = i;
            pm.t = mm.best;
            pm.d1 = mm.d1;
            pm.d2 = mm.d2;
            P.pairs[o] = pm;
        }
    }
}

// ---------------------------------------------------------------- host side
constexpr int kMatchMaxSplits = 64;
constexpr size_t kPlanBytes = 256;             // the published plan precedes the partials

int hamming_splits_alloc(int nt_cap) { return std::max(1, std::min(kMatchMaxSplits, (nt_cap + kMTile - 1) / kMTile)); }

size_t hamming_partial_bytes(int nq, int nt)
{
    return kPlanBytes + sizeof(uint2) * (size_t)hamming_splits_alloc(nt) * (size_t)std::max(nq, 1);
}

int pair_blocks(int nq) { return std::max(1, (nq + kPairBlock - 1) / kPairBlock); }

void match_problem_init(MatchProblem &P, const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                        const int32_t *d_nt, void *region, int s_alloc, asift_match *out, uint8_t *accept,
                        int32_t *n_acc)
{
    P = MatchProblem{};
    P.q = reinterpret_cast<const uint4 *>(q);
    P.t = reinterpret_cast<const uint4 *>(t);
    P.d_nq = d_nq;
    P.d_nt = d_nt;
    P.nq_cap = nq;
    P.nt_cap = nt;
    P.s_alloc = s_alloc > 0 ? s_alloc : hamming_splits_alloc(nt);
    P.plan = static_cast<int *>(region);
    P.part = reinterpret_cast<uint2 *>(static_cast<char *>(region) + kPlanBytes);
    P.out = out;
    P.accept = accept;
    P.n_acc = n_acc;
    P.n_blk = pair_blocks(nq);
}

void match_problems_offsets(MatchProblem *probs, int n, int *total_q, int *total_blk)
{
    int q = 0, b = 0;
    for (int i = 0; i < n; ++i) {
        probs[i].q_off = q;
        probs[i].blk_off = b;
        q += probs[i].nq_cap;
        b += probs[i].n_blk;
    }
    *total_q = q;
    *total_blk = b;
}

int match_max_problems() { return kMaxMatchProblems; }

cudaError_t launch_match(const MatchProblem *d_probs, int n_probs, const MatchProblem &single, int total_q,
                         bool any_train, int num, int den, const MatchTuning &tune, cudaStream_t s)
{
    if (total_q <= 0) return cudaSuccess;
    const int grid = tune.grid > 0 ? tune.grid : device_sm_count() * 7;
    const int target = tune.target_items > 0 ? tune.target_items : 2 * grid;
    if (any_train) {
        hamming_top2_kernel<<<grid, kMThreads, 0, s>>>(d_probs, n_probs, single, target);
        note_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_merge(d_probs, n_probs, single, total_q, num, den, s);
}

cudaError_t launch_merge(const MatchProblem *d_probs, int n_probs, const MatchProblem &single, int total_q, int num,
                         int den, cudaStream_t s)
{
    if (total_q <= 0) return cudaSuccess;
    merge_kernel<<<(total_q + 255) / 256, 256, 0, s>>>(d_probs, n_probs, single, total_q, num, den);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_hamming(const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                           const int32_t *d_nt, int num, int den, asift_match *out, uint8_t *accept,
                           int32_t *n_acc, void *part, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    MatchProblem P;
    match_problem_init(P, q, nq, d_nq, t, nt, d_nt, part, 0, out, accept, n_acc);
    return launch_match(nullptr, 0, P, nq, nt > 0, num, den, MatchTuning{}, s);
}

cudaError_t launch_pairs(const MatchProblem *d_probs, int n_probs, const MatchProblem &single, int total_blk,
                         int32_t *block_count, const DevLevel *lv, int nv, int32_t *status, cudaStream_t s)
{
    if (total_blk <= 0) return cudaSuccess;
    pair_count_kernel<<<total_blk, kPairBlock, 0, s>>>(d_probs, n_probs, single, block_count);
    pair_write_kernel<<<total_blk, kPairBlock, 0, s>>>(d_probs, n_probs, single, block_count, lv, nv, status);
    note_launch(2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- coarse stage: matches per view
// Best-parameter selection of Sec. III-B: the parameter group whose simulated
// view of the reference gathers the most accepted matches against the target.
// view_count_kernel histograms the accepted queries of one pool by the view
// they were detected in (shared-memory bins, one global add per bin and
// block); view_argmax_kernel (one block) takes the largest count, the lowest
// view index among equal counts.
constexpr int kCountBlock = 256;

__global__ void __launch_bounds__(kCountBlock)
view_count_kernel(const asift_keypoint *__restrict__ kp, const uint8_t *__restrict__ accept,
                  const int32_t *__restrict__ d_nq, int nq_cap, int view0, int n_views, int32_t *__restrict__ counts)
{
    extern __shared__ int bins[];
    for (int v = threadIdx.x; v < n_views; v += blockDim.x) bins[v] = 0;
    __syncthreads();
    const int nq = count_of(d_nq, nq_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        if (!accept[i]) continue;
        const int v = (int)kp[i].view - view0;
        if (v >= 0 && v < n_views) atomicAdd(&bins[v], 1);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < n_views; v += blockDim.x)
        if (bins[v]) atomicAdd(&counts[v], bins[v]);
}

__device__ __forceinline__ bool count_better(int c, int v, int bc, int bv) { return c > bc || (c == bc && v < bv); }

__global__ void __launch_bounds__(kCountBlock)
view_argmax_kernel(const int32_t *__restrict__ counts, int n_views, int32_t *__restrict__ best)
{
    __shared__ int sc[kCountBlock / 32], sv[kCountBlock / 32];
    int bc = -1, bv = n_views;
    for (int v = threadIdx.x; v < n_views; v += blockDim.x)
        if (count_better(counts[v], v, bc, bv)) { bc = counts[v]; bv = v; }
    for (int o = 16; o; o >>= 1) {
        const int c = __shfl_xor_sync(0xffffffffu, bc, o), v = __shfl_xor_sync(0xffffffffu, bv, o);
        if (count_better(c, v, bc, bv)) { bc = c; bv = v; }
    }
    if ((threadIdx.x & 31) == 0) { sc[threadIdx.x >> 5] = bc; sv[threadIdx.x >> 5] = bv; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kCountBlock / 32; ++w)
            if (count_better(sc[w], sv[w], bc, bv)) { bc = sc[w]; bv = sv[w]; }
        *best = bv;
    }
}

int view_count_max_views() { return 8192; }

cudaError_t launch_view_counts(const asift_keypoint *kp, const uint8_t *accept, const int32_t *d_nq, int nq_cap,
                               int view0, int n_views, int32_t *counts, int32_t *best, cudaStream_t s)
{
    if (n_views < 1 || n_views > view_count_max_views() || nq_cap < 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n_views, s);
    if (e != cudaSuccess) return e;
    if (nq_cap > 0) {
        const int grid = std::min((nq_cap + kCountBlock - 1) / kCountBlock, 2 * 152);
        view_count_kernel<<<grid, kCountBlock, sizeof(int) * (size_t)n_views, s>>>(kp, accept, d_nq, nq_cap, view0,
                                                                                 n_views, counts);
        note_launch();
    }
    if (best) {
        view_argmax_kernel<<<1, kCountBlock, 0, s>>>(counts, n_views, best);
        note_launch();
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- allocation-free matcher
// The partial keys of hamming_match_noalloc live in this file-scope array
// (ASIFT_NOALLOC_SCRATCH_BYTES per device that loads the library).  Host code
// must not pass the symbol itself to a kernel (on the host it names a host-side
// shadow, not device memory): its device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, and cached.
static __device__ __align__(256) unsigned char g_noalloc_part[ASIFT_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {};   // unique id of the context the address belongs to

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// The unique id of the calling thread's current CUDA context (0 when there is
// none yet or the driver does not tell: then the address is looked up again
// on every call): ids are never reused, so an address cached under one
// stays valid for exactly that context.
unsigned long long current_ctx_id()
{
    static CtxGetCurrentFn get_cur = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    static CtxGetIdFn get_id = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetIdFn>(p);
    }();
    void *c = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
    return id;
}
}  // namespace

// The device address of the fixed scratch array in the current context of
// the current device.  The first call in a context looks it up (a host-side
// query: no allocation, no work on any stream); later calls in the same
// context reuse it.  After cudaDeviceReset the device has a new context, so
// the next call looks the address up again.
static cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long id = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev] || id == 0 || g_noalloc_ctx[dev] != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_part);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
        g_noalloc_ctx[dev] = id;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

cudaError_t launch_hamming_noalloc(const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                                   const int32_t *d_nt, int num, int den, asift_match *out, uint8_t *accept,
                                   int32_t *n_acc, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    void *region = nullptr;
    cudaError_t e = noalloc_scratch(&region);
    if (e != cudaSuccess) return e;
    // as many train slices as the fixed array holds for nq queries (at least one)
    const long long entries = (long long)((ASIFT_NOALLOC_SCRATCH_BYTES - kPlanBytes) / sizeof(uint2));
    const int s_alloc = (int)std::max(1LL, std::min<long long>(hamming_splits_alloc(nt), entries / nq));
    MatchProblem P;
    match_problem_init(P, q, nq, d_nq, t, nt, d_nt, region, s_alloc, out, accept, n_acc);
    return launch_match(nullptr, 0, P, nq, nt > 0, num, den, MatchTuning{}, s);
}

}  // namespace asift
