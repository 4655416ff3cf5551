// match.cu -- brute-force Hamming matching with the ratio test (Sec. III-B,
// Sec. IV-C) on sm_103a, and the accepted-pair output of match_pair.
//
// hamming_top2_kernel: each thread keeps kMQ query descriptors (2 x uint4 each)
// in registers; the CTA stages kMTile train descriptors in shared memory and
// every thread scans them with XOR + popc.  The running nearest and
// second-nearest are kept as packed keys (distance << 23 | train index), so a
// min/max network gives the lowest index on distance ties and d2 counts equal
// distances.  The train set is split over gridDim.y slices; merge_kernel takes
// the two smallest keys over the slices (exact: keys are unique).
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace asift {

constexpr int kMQ = 4;
constexpr int kMThreads = 128;
constexpr int kMTile = 256;
constexpr unsigned kNoKey = 0xffffffffu;

// Hamming distance of two 256-bit descriptors.  The eight XOR words are summed
// bit-sliced with carry-save adders (three-input XOR and majority, one LOP3
// each), leaving four words of weight 1, 2, 4 and 8: four popc instead of
// eight, the popc pipe being the matcher's bottleneck.
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

// Split of the work into (query block, train slice) items, decided on the
// device from the actual counts so that a pool smaller than its capacity
// still fills the GPU.  Every CTA derives the same plan.
struct MatchPlan {
    int n_split, chunk;
};

__device__ __forceinline__ MatchPlan match_plan(int nq, int nt, int s_alloc, int target_items)
{
    MatchPlan p{0, kMTile};
    if (nq <= 0 || nt <= 0) return p;
    const int qblocks = (nq + kMThreads * kMQ - 1) / (kMThreads * kMQ);
    int s = max(1, (target_items + qblocks - 1) / qblocks);
    s = min(s, (nt + kMTile - 1) / kMTile);
    s = max(1, min(s, s_alloc));
    int chunk = (nt + s - 1) / s;
    chunk = ((chunk + kMTile - 1) / kMTile) * kMTile;
    p.chunk = chunk;
    p.n_split = (nt + chunk - 1) / chunk;
    return p;
}

// Persistent over the items: item = split * qblocks + query block.  The plan
// is published in plan_out (two ints) for the merge kernel.
__global__ void __launch_bounds__(kMThreads, 8)
hamming_top2_kernel(const uint4 *__restrict__ q, int nq_cap, const int32_t *__restrict__ d_nq,
                    const uint4 *__restrict__ t, int nt_cap, const int32_t *__restrict__ d_nt, int s_alloc,
                    int target_items, int *__restrict__ plan_out, uint2 *__restrict__ part)
{
    __shared__ uint4 st[2 * kMTile];
    const int nq = d_nq ? min(*d_nq, nq_cap) : nq_cap;
    const int nt = d_nt ? min(*d_nt, nt_cap) : nt_cap;
    const MatchPlan P = match_plan(nq, nt, s_alloc, target_items);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        plan_out[0] = P.n_split;
        plan_out[1] = P.chunk;
    }
    const int qblocks = (nq + kMThreads * kMQ - 1) / (kMThreads * kMQ);
    const int items = qblocks * P.n_split;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int split = item / qblocks, qb = item - split * qblocks;
        const int qbase = qb * (kMThreads * kMQ);
        const int t0 = split * P.chunk, t1 = min(nt, t0 + P.chunk);
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

__global__ void __launch_bounds__(256)
merge_kernel(const uint2 *__restrict__ part, const int *__restrict__ plan, int nq_cap,
             const int32_t *__restrict__ d_nq, int nt_cap, const int32_t *__restrict__ d_nt, int num, int den,
             asift_match *__restrict__ out, uint8_t *__restrict__ accept, int32_t *__restrict__ n_acc)
{
    const int nq = d_nq ? min(*d_nq, nq_cap) : nq_cap;
    const int nt = d_nt ? min(*d_nt, nt_cap) : nt_cap;
    const int n_split = (plan && nt > 0) ? plan[0] : 0;
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    bool acc = false;
    if (qi < nq) {
        unsigned b1 = kNoKey, b2 = kNoKey;
        for (int s = 0; s < n_split; ++s) {
            const uint2 p = part[(size_t)s * nq_cap + qi];
            b2 = min(b2, max(b1, p.x));
            b1 = min(b1, p.x);
            b2 = min(b2, max(b1, p.y));
            b1 = min(b1, p.y);
        }
        asift_match m;
        m.best = (b1 == kNoKey) ? -1 : (int)(b1 & 0x7fffffu);
        m.d1 = (uint16_t)((b1 == kNoKey) ? 257 : (b1 >> 23));
        m.d2 = (uint16_t)((b2 == kNoKey) ? 257 : (b2 >> 23));
        acc = nt >= 2 && den * (int)m.d1 < num * (int)m.d2;
        out[qi] = m;
        if (accept) accept[qi] = (uint8_t)acc;
    }
    if (n_acc) {
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        if ((threadIdx.x & 31) == 0 && bal) atomicAdd(n_acc, __popc(bal));
    }
}

// ---------------------------------------------------------------- accepted pairs
constexpr int kPairBlock = 1024;

__global__ void __launch_bounds__(kPairBlock)
pair_count_kernel(const uint8_t *__restrict__ accept, int nq_cap, const int32_t *__restrict__ d_nq,
                  int32_t *__restrict__ block_count)
{
    __shared__ int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int nq = min(*d_nq, nq_cap);
    const int i = blockIdx.x * kPairBlock + threadIdx.x;
    const bool a = i < nq && accept[i];
    const unsigned bal = __ballot_sync(0xffffffffu, a);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&s, __popc(bal));
    __syncthreads();
    if (threadIdx.x == 0) block_count[blockIdx.x] = s;
}

// Keypoint of view V at level l, position (x, y) -> source image pixel.
__device__ void backproject(const DevView &V, int l, int x, int y, float *sx, float *sy)
{
    long long p5 = 1, p6 = 1;
    for (int i = 0; i < l; ++i) { p5 *= 5; p6 *= 6; }
    const int Wl = (int)((2LL * V.Wv * p5 + p6) / (2 * p6));
    const int Hl = (int)((2LL * V.Hv * p5 + p6) / (2 * p6));
    const double x0 = (x + 0.5) * (double)V.Wv / (double)Wl - 0.5;
    const double y0 = (y + 0.5) * (double)V.Hv / (double)Hl - 0.5;
    const double X = V.t * (x0 - (V.Wv - 1) * 0.5) + (V.Wr - 1) * 0.5;
    const double dx = X - (V.Wr - 1) * 0.5, dy = y0 - (V.Hr - 1) * 0.5;
    *sx = (float)(V.cosd * dx + V.sind * dy + (V.W - 1) * 0.5);
    *sy = (float)(-V.sind * dx + V.cosd * dy + (V.H - 1) * 0.5);
}

__global__ void __launch_bounds__(kPairBlock)
pair_write_kernel(const uint8_t *__restrict__ accept, const asift_match *__restrict__ m, int nq_cap,
                  const int32_t *__restrict__ d_nq, const int32_t *__restrict__ block_count,
                  const asift_keypoint *__restrict__ kp1, const asift_keypoint *__restrict__ kp2,
                  const DevView *__restrict__ views, asift_pair_match *__restrict__ out, int cap,
                  int32_t *__restrict__ d_n, int32_t *__restrict__ status)
{
    __shared__ int wsum[kPairBlock / 32];
    __shared__ int base;
    const int nq = min(*d_nq, nq_cap);
    if (threadIdx.x == 0) {
        int b = 0;
        for (int k = 0; k < (int)blockIdx.x; ++k) b += block_count[k];
        base = b;
    }
    const int i = blockIdx.x * kPairBlock + threadIdx.x;
    const bool a = i < nq && accept[i];
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, a);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < kPairBlock / 32; ++k) { const int v = wsum[k]; wsum[k] = acc; acc += v; }
        if (blockIdx.x == gridDim.x - 1) {
            *d_n = base + acc;
            if (base + acc > cap) set_status(status, ASIFT_ERR_CAPACITY);
        }
    }
    __syncthreads();
    if (a) {
        const int o = base + wsum[w] + __popc(bal & ((1u << lane) - 1u));
        if (o < cap) {
            const asift_match mm = m[i];
            const asift_keypoint k1 = kp1[i], k2 = kp2[mm.best];
            asift_pair_match pm;
            backproject(views[k1.view], k1.level, k1.x, k1.y, &pm.x1, &pm.y1);
            backproject(views[k2.view], k2.level, k2.x, k2.y, &pm.x2, &pm.y2);
            pm.q = i;
            pm.t = mm.best;
            pm.d1 = mm.d1;
            pm.d2 = mm.d2;
            out[o] = pm;
        }
    }
}

// ---------------------------------------------------------------- host side
constexpr int kMatchMaxSplits = 64;
constexpr int kMatchGrid = 152 * 8;            // persistent CTAs (8 per SM at 64 registers)
constexpr int kMatchTargetItems = 2 * kMatchGrid;
constexpr size_t kPlanBytes = 256;             // the published plan precedes the partials

int hamming_splits_alloc(int nt_cap) { return std::max(1, std::min(kMatchMaxSplits, (nt_cap + kMTile - 1) / kMTile)); }

size_t hamming_partial_bytes(int nq, int nt)
{
    return kPlanBytes + sizeof(uint2) * (size_t)hamming_splits_alloc(nt) * (size_t)std::max(nq, 1);
}

static cudaError_t launch_match_kernels(const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                                        const int32_t *d_nt, int num, int den, asift_match *out, uint8_t *accept,
                                        int32_t *n_acc, void *region, int s_alloc, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    int *plan = static_cast<int *>(region);
    uint2 *part = reinterpret_cast<uint2 *>(static_cast<char *>(region) + kPlanBytes);
    if (nt > 0) {
        hamming_top2_kernel<<<kMatchGrid, kMThreads, 0, s>>>(reinterpret_cast<const uint4 *>(q), nq, d_nq,
                                                            reinterpret_cast<const uint4 *>(t), nt, d_nt, s_alloc,
                                                            kMatchTargetItems, plan, part);
        note_launch();
    }
    merge_kernel<<<(nq + 255) / 256, 256, 0, s>>>(part, nt > 0 ? plan : nullptr, nq, d_nq, nt, d_nt, num, den, out,
                                                  accept, n_acc);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_hamming(const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                           const int32_t *d_nt, int num, int den, asift_match *out, uint8_t *accept,
                           int32_t *n_acc, void *part, cudaStream_t s)
{
    return launch_match_kernels(q, nq, d_nq, t, nt, d_nt, num, den, out, accept, n_acc, part,
                                hamming_splits_alloc(nt), s);
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
}  // namespace

static cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_part);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
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
    return launch_match_kernels(q, nq, d_nq, t, nt, d_nt, num, den, out, accept, n_acc, region, s_alloc, s);
}

int pair_blocks(int nq) { return std::max(1, (nq + kPairBlock - 1) / kPairBlock); }

cudaError_t launch_pairs(const uint8_t *accept, const asift_match *m, int nq_cap, const int32_t *d_nq,
                         int32_t *block_count, const asift_keypoint *kp1, const asift_keypoint *kp2,
                         const DevView *views, asift_pair_match *out, int cap, int32_t *d_n, int32_t *status,
                         cudaStream_t s)
{
    const int nb = pair_blocks(nq_cap);
    pair_count_kernel<<<nb, kPairBlock, 0, s>>>(accept, nq_cap, d_nq, block_count);
    pair_write_kernel<<<nb, kPairBlock, 0, s>>>(accept, m, nq_cap, d_nq, block_count, kp1, kp2, views, out, cap, d_n,
                                                status);
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace asift
