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

__device__ __forceinline__ unsigned ham256(const uint4 &a0, const uint4 &a1, const uint4 &b0, const uint4 &b1)
{
    return __popc(a0.x ^ b0.x) + __popc(a0.y ^ b0.y) + __popc(a0.z ^ b0.z) + __popc(a0.w ^ b0.w) +
           __popc(a1.x ^ b1.x) + __popc(a1.y ^ b1.y) + __popc(a1.z ^ b1.z) + __popc(a1.w ^ b1.w);
}

__global__ void __launch_bounds__(kMThreads)
hamming_top2_kernel(const uint4 *__restrict__ q, int nq_cap, const int32_t *__restrict__ d_nq,
                    const uint4 *__restrict__ t, int nt_cap, const int32_t *__restrict__ d_nt, int chunk,
                    uint2 *__restrict__ part)
{
    __shared__ uint4 st[2 * kMTile];
    const int nq = d_nq ? min(*d_nq, nq_cap) : nq_cap;
    const int nt = d_nt ? min(*d_nt, nt_cap) : nt_cap;
    const int qbase = blockIdx.x * (kMThreads * kMQ);
    if (qbase >= nq) return;
    const int t0 = blockIdx.y * chunk, t1 = min(nt, t0 + chunk);

    uint4 qa[kMQ], qb[kMQ];
    unsigned b1[kMQ], b2[kMQ];
#pragma unroll
    for (int k = 0; k < kMQ; ++k) {
        const int qi = qbase + k * kMThreads + threadIdx.x;
        if (qi < nq) {
            qa[k] = q[2LL * qi];
            qb[k] = q[2LL * qi + 1];
        } else {
            qa[k] = make_uint4(0, 0, 0, 0);
            qb[k] = qa[k];
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
                const unsigned key = (ham256(qa[k], qb[k], x0, x1) << 23) | idx;
                b2[k] = min(b2[k], max(b1[k], key));
                b1[k] = min(b1[k], key);
            }
        }
    }
    if (t0 >= t1) return;
#pragma unroll
    for (int k = 0; k < kMQ; ++k) {
        const int qi = qbase + k * kMThreads + threadIdx.x;
        if (qi < nq) part[(size_t)blockIdx.y * nq_cap + qi] = make_uint2(b1[k], b2[k]);
    }
}

__global__ void __launch_bounds__(256)
merge_kernel(const uint2 *__restrict__ part, int n_split, int chunk, int nq_cap, const int32_t *__restrict__ d_nq,
             int nt_cap, const int32_t *__restrict__ d_nt, int num, int den, asift_match *__restrict__ out,
             uint8_t *__restrict__ accept, int32_t *__restrict__ n_acc)
{
    const int nq = d_nq ? min(*d_nq, nq_cap) : nq_cap;
    const int nt = d_nt ? min(*d_nt, nt_cap) : nt_cap;
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    bool acc = false;
    if (qi < nq) {
        unsigned b1 = kNoKey, b2 = kNoKey;
        for (int s = 0; s < n_split; ++s) {
            if (s * chunk >= nt) break;
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
void hamming_plan(int nq, int nt, int *n_split, int *chunk)
{
    const int qblocks = std::max(1, (nq + kMThreads * kMQ - 1) / (kMThreads * kMQ));
    const int target = 152 * 6;                     // CTAs in flight over the 152 SMs
    int s = std::max(1, (target + qblocks - 1) / qblocks);
    const int max_s = std::max(1, (nt + kMTile - 1) / kMTile);
    s = std::min(s, max_s);
    int c = (nt + s - 1) / s;
    c = ((c + kMTile - 1) / kMTile) * kMTile;       // whole train tiles per slice
    if (c <= 0) c = kMTile;
    *chunk = c;
    *n_split = std::max(1, (nt + c - 1) / c);
}

size_t hamming_partial_bytes(int nq, int nt)
{
    int s, c;
    hamming_plan(nq, nt, &s, &c);
    return sizeof(uint2) * (size_t)s * (size_t)std::max(nq, 1);
}

cudaError_t launch_hamming(const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                           const int32_t *d_nt, int num, int den, asift_match *out, uint8_t *accept,
                           int32_t *n_acc, void *part, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    int n_split, chunk;
    hamming_plan(nq, nt, &n_split, &chunk);
    if (nt > 0) {
        dim3 grid((nq + kMThreads * kMQ - 1) / (kMThreads * kMQ), n_split);
        hamming_top2_kernel<<<grid, kMThreads, 0, s>>>(reinterpret_cast<const uint4 *>(q), nq, d_nq,
                                                      reinterpret_cast<const uint4 *>(t), nt, d_nt, chunk,
                                                      static_cast<uint2 *>(part));
        note_launch();
    }
    merge_kernel<<<(nq + 255) / 256, 256, 0, s>>>(static_cast<const uint2 *>(part), nt > 0 ? n_split : 0, chunk, nq,
                                                  d_nq, nt, d_nt, num, den, out, accept, n_acc);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- allocation-free matcher
// The partial keys of hamming_match_noalloc live in this file-scope array
// (ASIFT_NOALLOC_SCRATCH_BYTES per device that loads the library).  Host code
// must not pass the symbol itself to a kernel (on the host it names a host-side
// shadow, not device memory): its device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, and cached.
static __device__ __align__(256) uint2 g_noalloc_part[ASIFT_NOALLOC_SCRATCH_BYTES / sizeof(uint2)];

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
    void *part = nullptr;
    cudaError_t e = noalloc_scratch(&part);
    if (e != cudaSuccess) return e;
    const long long cap = (long long)(ASIFT_NOALLOC_SCRATCH_BYTES / sizeof(uint2));
    int n_split, chunk;
    hamming_plan(nq, nt, &n_split, &chunk);
    if ((long long)n_split * nq > cap) {          // fewer, longer train slices
        const int s_max = (int)std::max(1LL, cap / nq);
        chunk = (nt + s_max - 1) / s_max;
        chunk = ((chunk + kMTile - 1) / kMTile) * kMTile;
        if (chunk <= 0) chunk = kMTile;
        n_split = std::max(1, (nt + chunk - 1) / chunk);
    }
    if (nt > 0) {
        dim3 grid((nq + kMThreads * kMQ - 1) / (kMThreads * kMQ), n_split);
        hamming_top2_kernel<<<grid, kMThreads, 0, s>>>(reinterpret_cast<const uint4 *>(q), nq, d_nq,
                                                      reinterpret_cast<const uint4 *>(t), nt, d_nt, chunk,
                                                      static_cast<uint2 *>(part));
        note_launch();
    }
    merge_kernel<<<(nq + 255) / 256, 256, 0, s>>>(static_cast<const uint2 *>(part), nt > 0 ? n_split : 0, chunk, nq,
                                                  d_nq, nt, d_nt, num, den, out, accept, n_acc);
    note_launch();
    return cudaGetLastError();
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
