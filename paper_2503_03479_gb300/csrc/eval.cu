// eval.cu -- evaluation of the accepted pairs on sm_103a: duplicate removal
// in original coordinates, the precision count of Eq. (5)-(6), a homography
// by RANSAC [28] (Sec. III-C) and its inliers (Eq. (7)).
//
//   1. dedup_insert_kernel / dedup_keep_kernel: a pair's key is the nearest
//      pixels of (x1, y1, x2, y2) (floor(x + 1/2) in fp32).  An open-addressing
//      table keyed by the pair index holds, per key, the smallest index with
//      that key (insert by compare-and-swap, then atomicMin; any index held
//      has the slot's key, so comparisons recompute it).  A pair is kept iff
//      it is its key's smallest index: the earliest of each duplicate group.
//   2. block_count_kernel / compact_kernel: order-preserving compaction of the
//      kept pairs.
//   3. precision_kernel: pairs within sqrt(th_sq) of the true mapping.
//   4. ransac_fit_kernel: one thread per hypothesis draws its four pairs
//      (caller's random numbers mod n) and solves the 8x8 system by Gaussian
//      elimination with partial pivoting.
//   5. ransac_count_kernel: hypotheses x pairs, eight hypotheses per CTA
//      staged in shared memory; each test is decided in fp32 with an error
//      bound, in fp64 only within the bound of the threshold.
//   6. ransac_best_kernel (the largest count, the lowest hypothesis on ties)
//      and inlier_kernel.
// Every fp64 step is one IEEE operation (the _rn intrinsics are never fused),
// so each decision is taken on exactly the values the written order gives.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace asift {

constexpr int kEvalBlock = 256;
constexpr int kHypPerCta = 8;
constexpr int kEmpty = -1;

__device__ __forceinline__ int pix_of(float x) { return (int)floorf(__fadd_rn(x, 0.5f)); }

struct PairKey4 {
    int a, b, c, d;
};

__device__ __forceinline__ PairKey4 key_of(const asift_pair_match &p)
{
    return PairKey4{pix_of(p.x1), pix_of(p.y1), pix_of(p.x2), pix_of(p.y2)};
}

__device__ __forceinline__ bool same_key(const PairKey4 &u, const PairKey4 &v)
{
    return u.a == v.a && u.b == v.b && u.c == v.c && u.d == v.d;
}

__device__ __forceinline__ unsigned hash_key(const PairKey4 &k)
{
    unsigned h = (unsigned)k.a * 0x9E3779B1u;
    h = (h ^ (h >> 15)) + (unsigned)k.b * 0x85EBCA77u;
    h = (h ^ (h >> 13)) + (unsigned)k.c * 0xC2B2AE3Du;
    h = (h ^ (h >> 16)) + (unsigned)k.d * 0x27D4EB2Fu;
    return h ^ (h >> 15);
}

__device__ __forceinline__ int pair_count(const int32_t *d_n, int cap) { return min(max(*d_n, 0), cap); }

__global__ void __launch_bounds__(kEvalBlock)
dedup_insert_kernel(const asift_pair_match *__restrict__ pairs, const int32_t *__restrict__ d_n, int cap,
                    int *__restrict__ table, unsigned tmask, asift_eval_result *__restrict__ res)
{
    const int n = pair_count(d_n, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const PairKey4 k = key_of(pairs[i]);
        unsigned s = hash_key(k) & tmask;
        bool done = false;
        // the table has at least twice as many slots as pairs: a free slot or
        // the key's slot is always reached within tmask + 1 probes
        for (unsigned probe = 0; probe <= tmask && !done; ++probe, s = (s + 1) & tmask) {
            const int prev = atomicCAS(&table[s], kEmpty, i);
            if (prev == kEmpty) {
                done = true;
            } else if (same_key(key_of(pairs[prev]), k)) {
                atomicMin(&table[s], i);
                done = true;
            }
        }
        if (!done) res->status = ASIFT_ERR_CAPACITY;
    }
}

__global__ void __launch_bounds__(kEvalBlock)
dedup_keep_kernel(const asift_pair_match *__restrict__ pairs, const int32_t *__restrict__ d_n, int cap,
                  const int *__restrict__ table, unsigned tmask, uint8_t *__restrict__ keep)
{
    const int n = pair_count(d_n, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const PairKey4 k = key_of(pairs[i]);
        unsigned s = hash_key(k) & tmask;
        int owner = i;
        for (unsigned probe = 0; probe <= tmask; ++probe, s = (s + 1) & tmask) {
            const int v = table[s];
            if (v == kEmpty) break;           // not reached: the pair itself was inserted
            if (same_key(key_of(pairs[v]), k)) {
                owner = v;
                break;
            }
        }
        keep[i] = (uint8_t)(owner == i);
    }
}

// Kept pairs per block of kEvalBlock pairs, then each block writes its kept
// pairs after those of the blocks before it.
__global__ void __launch_bounds__(kEvalBlock)
block_count_kernel(const int32_t *__restrict__ d_n, int cap, const uint8_t *__restrict__ keep,
                   int32_t *__restrict__ block_count)
{
    __shared__ int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int n = pair_count(d_n, cap);
    const int i = blockIdx.x * kEvalBlock + threadIdx.x;
    const unsigned bal = __ballot_sync(0xffffffffu, i < n && keep[i]);
    if ((threadIdx.x & 31u) == 0 && bal) atomicAdd(&s, __popc(bal));
    __syncthreads();
    if (threadIdx.x == 0) block_count[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kEvalBlock)
compact_kernel(const asift_pair_match *__restrict__ pairs, const int32_t *__restrict__ d_n, int cap,
               const uint8_t *__restrict__ keep, const int32_t *__restrict__ block_count,
               asift_pair_match *__restrict__ out, asift_eval_result *__restrict__ res)
{
    __shared__ int wsum[kEvalBlock / 32];
    __shared__ int base;
    const int n = pair_count(d_n, cap);
    if (threadIdx.x == 0) {
        int b = 0;
        for (int k = 0; k < (int)blockIdx.x; ++k) b += block_count[k];
        base = b;
    }
    const int i = blockIdx.x * kEvalBlock + threadIdx.x;
    const bool a = i < n && keep[i];
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, a);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < kEvalBlock / 32; ++k) {
            const int v = wsum[k];
            wsum[k] = acc;
            acc += v;
        }
        if (blockIdx.x == gridDim.x - 1) {
            res->n_pairs = n;
            res->n_unique = base + acc;
        }
    }
    __syncthreads();
    if (a) out[base + wsum[w] + __popc(bal & ((1u << lane) - 1u))] = pairs[i];
}

// Squared distance between H (x, y) and (u, v), one rounding per operation
// in the order ((h0 x + h1 y) + h2) / ((h6 x + h7 y) + h8) - u, ...
__device__ __forceinline__ double reproj_sq(const double *H, double x, double y, double u, double v)
{
    const double X = __dadd_rn(__dadd_rn(__dmul_rn(H[0], x), __dmul_rn(H[1], y)), H[2]);
    const double Y = __dadd_rn(__dadd_rn(__dmul_rn(H[3], x), __dmul_rn(H[4], y)), H[5]);
    const double Z = __dadd_rn(__dadd_rn(__dmul_rn(H[6], x), __dmul_rn(H[7], y)), H[8]);
    const double dx = __dsub_rn(__ddiv_rn(X, Z), u), dy = __dsub_rn(__ddiv_rn(Y, Z), v);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

struct Hom9 {
    double h[9];
};

__device__ __forceinline__ int block_sum(int v)
{
    __shared__ int ws[kEvalBlock / 32];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31u) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kEvalBlock / 32; ++k) t += ws[k];
    __syncthreads();
    return t;                                   // valid in thread 0
}

__global__ void __launch_bounds__(kEvalBlock)
precision_kernel(const asift_pair_match *__restrict__ up, const Hom9 Ht, double th_sq,
                 asift_eval_result *__restrict__ res)
{
    const int n = res->n_unique;
    int c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const asift_pair_match p = up[i];
        c += reproj_sq(Ht.h, p.x1, p.y1, p.x2, p.y2) <= th_sq;
    }
    const int t = block_sum(c);
    if (threadIdx.x == 0 && t) atomicAdd(&res->r_num, t);
}

// Homography from four correspondences with h8 = 1 (eight linear equations,
// Gaussian elimination with partial pivoting: the first row with the largest
// |entry|; a pivot at most 1e-10 times the largest |entry| is degenerate).
__device__ bool homography4(const double *x, const double *y, const double *u, const double *v, double *H)
{
    double A[8][9];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double *r0 = A[2 * k], *r1 = A[2 * k + 1];
        r0[0] = x[k]; r0[1] = y[k]; r0[2] = 1.0; r0[3] = 0.0; r0[4] = 0.0; r0[5] = 0.0;
        r0[6] = -__dmul_rn(x[k], u[k]); r0[7] = -__dmul_rn(y[k], u[k]); r0[8] = u[k];
        r1[0] = 0.0; r1[1] = 0.0; r1[2] = 0.0; r1[3] = x[k]; r1[4] = y[k]; r1[5] = 1.0;
        r1[6] = -__dmul_rn(x[k], v[k]); r1[7] = -__dmul_rn(y[k], v[k]); r1[8] = v[k];
    }
    double amax = 0.0;
    for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 8; ++c) amax = fmax(amax, fabs(A[r][c]));
    const double tiny = __dmul_rn(1e-10, amax);
    for (int k = 0; k < 8; ++k) {
        int p = k;
        for (int r = k + 1; r < 8; ++r)
            if (fabs(A[r][k]) > fabs(A[p][k])) p = r;
        if (!(fabs(A[p][k]) > tiny)) return false;
        if (p != k)
            for (int c = 0; c < 9; ++c) {
                const double t = A[k][c];
                A[k][c] = A[p][c];
                A[p][c] = t;
            }
        for (int r = k + 1; r < 8; ++r) {
            const double f = __ddiv_rn(A[r][k], A[k][k]);
            for (int c = k + 1; c < 9; ++c) A[r][c] = __dsub_rn(A[r][c], __dmul_rn(f, A[k][c]));
            A[r][k] = 0.0;
        }
    }
    double h[8];
    for (int k = 7; k >= 0; --k) {
        double s = A[k][8];
        for (int c = k + 1; c < 8; ++c) s = __dsub_rn(s, __dmul_rn(A[k][c], h[c]));
        h[k] = __ddiv_rn(s, A[k][k]);
    }
    for (int k = 0; k < 8; ++k) {
        if (!isfinite(h[k])) return false;
        H[k] = h[k];
    }
    H[8] = 1.0;
    return true;
}

__global__ void __launch_bounds__(32)
ransac_fit_kernel(const asift_pair_match *__restrict__ up, const uint32_t *__restrict__ rnd, int n_hyp,
                  double *__restrict__ Hs, int32_t *__restrict__ counts, const asift_eval_result *__restrict__ res)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n_hyp) return;
    const int n = res->n_unique;
    double *Hh = Hs + 9 * (size_t)h;
    for (int c = 0; c < 9; ++c) Hh[c] = 0.0;
    counts[h] = -1;
    if (n < 4) return;
    int idx[4];
    for (int k = 0; k < 4; ++k) idx[k] = (int)(rnd[4 * (size_t)h + k] % (uint32_t)n);
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
            if (idx[a] == idx[b]) return;
    double xs[4], ys[4], us[4], vs[4];
    for (int k = 0; k < 4; ++k) {
        const asift_pair_match p = up[idx[k]];
        xs[k] = p.x1;
        ys[k] = p.y1;
        us[k] = p.x2;
        vs[k] = p.y2;
    }
    double H[9];
    if (!homography4(xs, ys, us, vs, H)) return;
    for (int c = 0; c < 9; ++c) Hh[c] = H[c];
    counts[h] = 0;
}

// The threshold test of one pair, decided as reproj_sq(H, ...) <= th_sq is,
// but mostly in fp32: an fp32 evaluation with a rigorous error bound decides
// every pair whose distance is clearly inside or outside the threshold, and
// only pairs within the bound of it take the fp64 path.  With unit roundoff
// u = 2^-24, the rounding of H to fp32 and the products and sums leave |X32 -
// X| <= 4u SX (SX = |h0 x| + |h1 y| + |h2|), likewise for Y and Z; the
// quotient and the difference add a few u more.  The bound below takes 16u
// (four times that) and rejects near-zero denominators, so a decision taken
// in fp32 is the fp64 decision.
// The rare undecided case, out of line so the fp32 loop stays small.
__device__ __noinline__ bool within_threshold_exact(const double *Hd, float x, float y, float u, float v, double th_sq)
{
    return reproj_sq(Hd, x, y, u, v) <= th_sq;
}

__device__ __forceinline__ bool within_threshold(const double *Hd, const float *Hf, float x, float y, float u, float v,
                                                 double th_sq, float th_lo, float th_hi)
{
    constexpr float kU = 16.0f / 16777216.0f;
    const float a0 = Hf[0] * x, a1 = Hf[1] * y, b0 = Hf[3] * x, b1 = Hf[4] * y, c0 = Hf[6] * x, c1 = Hf[7] * y;
    const float X = (a0 + a1) + Hf[2], Y = (b0 + b1) + Hf[5], Z = (c0 + c1) + Hf[8];
    const float SX = fabsf(a0) + fabsf(a1) + fabsf(Hf[2]);
    const float SY = fabsf(b0) + fabsf(b1) + fabsf(Hf[5]);
    const float SZ = fabsf(c0) + fabsf(c1) + fabsf(Hf[8]);
    if (fabsf(Z) > 4.0f * kU * SZ) {
        const float iz = 1.0f / Z;
        const float px = X * iz, py = Y * iz;
        const float dx = fabsf(px - u), dy = fabsf(py - v);
        const float ex = kU * ((SX + fabsf(px) * SZ) * fabsf(iz) + fabsf(px) + fabsf(u));
        const float ey = kU * ((SY + fabsf(py) * SZ) * fabsf(iz) + fabsf(py) + fabsf(v));
        const float hx = dx + ex, hy = dy + ey;
        const float lx = fmaxf(dx - ex, 0.f), ly = fmaxf(dy - ey, 0.f);
        if (hx * hx + hy * hy < th_lo) return true;      // NaN and infinity fall through
        if (lx * lx + ly * ly > th_hi) return false;
    }
    return within_threshold_exact(Hd, x, y, u, v, th_sq);
}

__global__ void __launch_bounds__(kEvalBlock)
ransac_count_kernel(const asift_pair_match *__restrict__ up, int n_hyp, const double *__restrict__ Hs,
                    int32_t *__restrict__ counts, const asift_eval_result *__restrict__ res)
{
    __shared__ double sH[kHypPerCta][9];
    __shared__ float sHf[kHypPerCta][9];
    __shared__ int sv[kHypPerCta];
    const int h0 = blockIdx.x * kHypPerCta;
    for (int k = threadIdx.x; k < kHypPerCta * 9; k += blockDim.x) {
        const int h = h0 + k / 9;
        const double hv = h < n_hyp ? Hs[9 * (size_t)h + k % 9] : 0.0;
        sH[k / 9][k % 9] = hv;
        sHf[k / 9][k % 9] = (float)hv;
    }
    if (threadIdx.x < kHypPerCta) {
        const int h = h0 + (int)threadIdx.x;
        sv[threadIdx.x] = h < n_hyp && counts[h] >= 0;
    }
    __syncthreads();
    const int n = res->n_unique;
    const double th_sq = res->ransac_th_sq;
    // fp32 thresholds strictly inside / outside th_sq by more than their own rounding
    const float th_lo = (float)th_sq * (1.0f - 1e-5f), th_hi = (float)th_sq * (1.0f + 1e-5f);
    int c[kHypPerCta];
#pragma unroll
    for (int k = 0; k < kHypPerCta; ++k) c[k] = 0;
    // the CTAs of one hypothesis group stride over the kept pairs together
    for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) {
        const asift_pair_match p = up[i];
#pragma unroll
        for (int k = 0; k < kHypPerCta; ++k)
            if (sv[k]) c[k] += within_threshold(sH[k], sHf[k], p.x1, p.y1, p.x2, p.y2, th_sq, th_lo, th_hi);
    }
#pragma unroll
    for (int k = 0; k < kHypPerCta; ++k) {
        const int t = block_sum(c[k]);
        if (threadIdx.x == 0 && sv[k] && t) atomicAdd(&counts[h0 + k], t);
    }
}

__device__ __forceinline__ bool hyp_better(int c, int h, int bc, int bh) { return c > bc || (c == bc && h < bh); }

__global__ void __launch_bounds__(kEvalBlock)
ransac_best_kernel(const int32_t *__restrict__ counts, int n_hyp, const double *__restrict__ Hs,
                   asift_eval_result *__restrict__ res)
{
    __shared__ int sc[kEvalBlock / 32], sh[kEvalBlock / 32];
    int bc = -1, bh = n_hyp;
    for (int h = threadIdx.x; h < n_hyp; h += blockDim.x)
        if (counts[h] >= 0 && hyp_better(counts[h], h, bc, bh)) {
            bc = counts[h];
            bh = h;
        }
    for (int o = 16; o; o >>= 1) {
        const int c = __shfl_xor_sync(0xffffffffu, bc, o), h = __shfl_xor_sync(0xffffffffu, bh, o);
        if (hyp_better(c, h, bc, bh)) {
            bc = c;
            bh = h;
        }
    }
    if ((threadIdx.x & 31u) == 0) {
        sc[threadIdx.x >> 5] = bc;
        sh[threadIdx.x >> 5] = bh;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kEvalBlock / 32; ++w)
            if (hyp_better(sc[w], sh[w], bc, bh)) {
                bc = sc[w];
                bh = sh[w];
            }
        const bool any = bc >= 0;
        res->best_hyp = any ? bh : -1;
        for (int c = 0; c < 9; ++c) res->H[c] = any ? Hs[9 * (size_t)bh + c] : 0.0;
    }
}

__global__ void __launch_bounds__(kEvalBlock)
inlier_kernel(const asift_pair_match *__restrict__ up, int cap, uint8_t *__restrict__ inlier,
              asift_eval_result *__restrict__ res)
{
    const int n = res->n_unique;
    const bool any = res->best_hyp >= 0;
    double H[9];
    for (int c = 0; c < 9; ++c) H[c] = res->H[c];
    int cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        bool in = false;
        if (i < n && any) {
            const asift_pair_match p = up[i];
            in = reproj_sq(H, p.x1, p.y1, p.x2, p.y2) <= res->ransac_th_sq;
        }
        if (inlier) inlier[i] = (uint8_t)in;
        cnt += in;
    }
    const int t = block_sum(cnt);
    if (threadIdx.x == 0 && t) atomicAdd(&res->n_inliers, t);
}

__global__ void eval_init_kernel(asift_eval_result *res, int r_num, double ransac_th_sq)
{
    if (threadIdx.x == 0) {
        res->n_pairs = 0;
        res->n_unique = 0;
        res->r_num = r_num;
        res->best_hyp = -1;
        res->n_inliers = 0;
        res->status = ASIFT_OK;
        res->ransac_th_sq = ransac_th_sq;
    }
    if (threadIdx.x < 9) res->H[threadIdx.x] = 0.0;
}

// ---------------------------------------------------------------- host side
static unsigned table_slots(int cap)
{
    unsigned t = 64;
    while (t < 2u * (unsigned)std::max(cap, 1)) t <<= 1;
    return t;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t eval_workspace_bytes(int cap, int n_hyp)
{
    const size_t blocks = (size_t)std::max(1, (cap + kEvalBlock - 1) / kEvalBlock);
    return align256(sizeof(int) * table_slots(cap)) + align256((size_t)std::max(cap, 1)) +
           align256(sizeof(int32_t) * blocks) + align256(sizeof(double) * 9 * (size_t)std::max(n_hyp, 1)) +
           align256(sizeof(int32_t) * (size_t)std::max(n_hyp, 1));
}

cudaError_t launch_eval(const asift_pair_match *d_pairs, const int32_t *d_n, int cap, const double *h_H_true,
                        double th_sq, const uint32_t *d_rnd, int n_hyp, double ransac_th_sq,
                        asift_pair_match *d_unique, uint8_t *d_inlier, int32_t *d_hyp_counts,
                        asift_eval_result *d_res, void *d_ws, cudaStream_t s)
{
    const unsigned slots = table_slots(cap);
    const int blocks = std::max(1, (cap + kEvalBlock - 1) / kEvalBlock);
    char *w = static_cast<char *>(d_ws);
    int *table = reinterpret_cast<int *>(w);
    w += align256(sizeof(int) * slots);
    uint8_t *keep = reinterpret_cast<uint8_t *>(w);
    w += align256((size_t)std::max(cap, 1));
    int32_t *bcount = reinterpret_cast<int32_t *>(w);
    w += align256(sizeof(int32_t) * blocks);
    double *Hs = reinterpret_cast<double *>(w);
    w += align256(sizeof(double) * 9 * (size_t)std::max(n_hyp, 1));
    int32_t *counts = d_hyp_counts ? d_hyp_counts : reinterpret_cast<int32_t *>(w);

    eval_init_kernel<<<1, 32, 0, s>>>(d_res, h_H_true ? 0 : -1, ransac_th_sq);
    note_launch();
    cudaError_t e = cudaMemsetAsync(table, 0xff, sizeof(int) * slots, s);
    if (e != cudaSuccess) return e;
    const int grid = std::min(blocks, 4 * 152);
    dedup_insert_kernel<<<grid, kEvalBlock, 0, s>>>(d_pairs, d_n, cap, table, slots - 1, d_res);
    dedup_keep_kernel<<<grid, kEvalBlock, 0, s>>>(d_pairs, d_n, cap, table, slots - 1, keep);
    block_count_kernel<<<blocks, kEvalBlock, 0, s>>>(d_n, cap, keep, bcount);
    compact_kernel<<<blocks, kEvalBlock, 0, s>>>(d_pairs, d_n, cap, keep, bcount, d_unique, d_res);
    note_launch(4);
    if (h_H_true) {
        Hom9 Ht;
        for (int c = 0; c < 9; ++c) Ht.h[c] = h_H_true[c];
        precision_kernel<<<grid, kEvalBlock, 0, s>>>(d_unique, Ht, th_sq, d_res);
        note_launch();
    }
    if (n_hyp > 0) {
        ransac_fit_kernel<<<(n_hyp + 31) / 32, 32, 0, s>>>(d_unique, d_rnd, n_hyp, Hs, counts, d_res);
        // hypothesis groups x CTAs per group: about two CTAs per SM, no more
        // CTAs per group than the capacity's blocks of pairs
        const int hyp_blocks = (n_hyp + kHypPerCta - 1) / kHypPerCta;
        const int gy = std::max(1, std::min((2 * 152 + hyp_blocks - 1) / hyp_blocks, blocks));
        ransac_count_kernel<<<dim3(hyp_blocks, gy), kEvalBlock, 0, s>>>(d_unique, n_hyp, Hs, counts, d_res);
        ransac_best_kernel<<<1, kEvalBlock, 0, s>>>(counts, n_hyp, Hs, d_res);
        note_launch(3);
    }
    inlier_kernel<<<grid, kEvalBlock, 0, s>>>(d_unique, cap, d_inlier, d_res);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asift
