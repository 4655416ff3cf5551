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
// Each launch serves a list of problems (one per image pair: all pairs of a
// plan, or one pair passed by value), so a batch costs one launch per stage.
// Also here: the scaling coefficient of Eq. (1) (Sec. III-A), a fixed-order
// fp64 reduction over consecutive pairs.
#include <algorithm>
#include <cmath>
#include <vector>

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

// One evaluation problem (the accepted pairs of one image pair) and its
// scratch.  A launch serves a list of problems: the pair-parallel kernels run
// blk_off .. blk_off + n_blk - 1 of a common block range, the per-hypothesis
// ones take the problem from blockIdx.z (or .y) and the per-problem ones
// from blockIdx.x.  A single problem can also be passed by value.
struct EvalProblem {
    const asift_pair_match *pairs;
    const int32_t *d_n;
    int cap;
    int blk_off, n_blk;           // blocks of kEvalBlock pairs
    unsigned tmask;               // table slots - 1
    int *table;
    uint8_t *keep;
    int32_t *bcount;
    asift_pair_match *unique;
    uint8_t *inlier;              // may be null
    double *Hs;
    int32_t *counts;
    asift_eval_result *res;
    int has_H;
    double Ht[9];
};

__device__ __forceinline__ const EvalProblem &eprob(const EvalProblem *many, const EvalProblem &single, int p)
{
    return many ? many[p] : single;
}

__device__ __forceinline__ int eval_problem_of_block(const EvalProblem *many, int n, int block)
{
    if (!many) return 0;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (many[mid].blk_off <= block) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void eval_init_kernel(const EvalProblem *__restrict__ many, const EvalProblem single, double ransac_th_sq)
{
    const EvalProblem &P = eprob(many, single, blockIdx.x);
    asift_eval_result *res = P.res;
    if (threadIdx.x == 0) {
        res->n_pairs = 0;
        res->n_unique = 0;
        res->r_num = P.has_H ? 0 : -1;
        res->best_hyp = -1;
        res->n_inliers = 0;
        res->status = ASIFT_OK;
        res->ransac_th_sq = ransac_th_sq;
    }
    if (threadIdx.x < 9) res->H[threadIdx.x] = 0.0;
    for (unsigned s = threadIdx.x; s <= P.tmask; s += blockDim.x) P.table[s] = kEmpty;
}

__global__ void __launch_bounds__(kEvalBlock)
dedup_insert_kernel(const EvalProblem *__restrict__ many, int n_probs, const EvalProblem single)
{
    const EvalProblem &P = eprob(many, single, eval_problem_of_block(many, n_probs, blockIdx.x));
    const int n = pair_count(P.d_n, P.cap);
    const int i = (blockIdx.x - P.blk_off) * kEvalBlock + threadIdx.x;
    if (i >= n) return;
    const asift_pair_match *__restrict__ pairs = P.pairs;
    int *__restrict__ table = P.table;
    const unsigned tmask = P.tmask;
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
    if (!done) P.res->status = ASIFT_ERR_CAPACITY;
}

__global__ void __launch_bounds__(kEvalBlock)
dedup_keep_kernel(const EvalProblem *__restrict__ many, int n_probs, const EvalProblem single)
{
    const EvalProblem &P = eprob(many, single, eval_problem_of_block(many, n_probs, blockIdx.x));
    const int n = pair_count(P.d_n, P.cap);
    const int i = (blockIdx.x - P.blk_off) * kEvalBlock + threadIdx.x;
    if (i >= n) return;
    const PairKey4 k = key_of(P.pairs[i]);
    unsigned s = hash_key(k) & P.tmask;
    int owner = i;
    for (unsigned probe = 0; probe <= P.tmask; ++probe, s = (s + 1) & P.tmask) {
        const int v = P.table[s];
        if (v == kEmpty) break;               // not reached: the pair itself was inserted
        if (same_key(key_of(P.pairs[v]), k)) {
            owner = v;
            break;
        }
    }
    P.keep[i] = (uint8_t)(owner == i);
}

// Kept pairs per block of kEvalBlock pairs, then each block writes its kept
// pairs after those of its problem's blocks before it.
__global__ void __launch_bounds__(kEvalBlock)
block_count_kernel(const EvalProblem *__restrict__ many, int n_probs, const EvalProblem single)
{
    __shared__ int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const EvalProblem &P = eprob(many, single, eval_problem_of_block(many, n_probs, blockIdx.x));
    const int n = pair_count(P.d_n, P.cap);
    const int lb = blockIdx.x - P.blk_off;
    const int i = lb * kEvalBlock + threadIdx.x;
    const unsigned bal = __ballot_sync(0xffffffffu, i < n && P.keep[i]);
    if ((threadIdx.x & 31u) == 0 && bal) atomicAdd(&s, __popc(bal));
    __syncthreads();
    if (threadIdx.x == 0) P.bcount[lb] = s;
}

__global__ void __launch_bounds__(kEvalBlock)
compact_kernel(const EvalProblem *__restrict__ many, int n_probs, const EvalProblem single)
{
    __shared__ int wsum[kEvalBlock / 32];
    __shared__ int base;
    const EvalProblem &P = eprob(many, single, eval_problem_of_block(many, n_probs, blockIdx.x));
    const int n = pair_count(P.d_n, P.cap);
    const int lb = blockIdx.x - P.blk_off;
    if (threadIdx.x == 0) {
        int b = 0;
        for (int k = 0; k < lb; ++k) b += P.bcount[k];
        base = b;
    }
    const int i = lb * kEvalBlock + threadIdx.x;
    const bool a = i < n && P.keep[i];
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
        if (lb == P.n_blk - 1) {
            P.res->n_pairs = n;
            P.res->n_unique = base + acc;
        }
    }
    __syncthreads();
    if (a) P.unique[base + wsum[w] + __popc(bal & ((1u << lane) - 1u))] = P.pairs[i];
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

// Eq. (6) over the kept pairs: every block of the problem's range takes a
// stride of them.
__global__ void __launch_bounds__(kEvalBlock)
precision_kernel(const EvalProblem *__restrict__ many, int n_probs, const EvalProblem single, double th_sq)
{
    const EvalProblem &P = eprob(many, single, eval_problem_of_block(many, n_probs, blockIdx.x));
    if (!P.has_H) return;                       // uniform over the block
    const int n = P.res->n_unique;
    int c = 0;
    for (int i = (blockIdx.x - P.blk_off) * kEvalBlock + threadIdx.x; i < n; i += P.n_blk * kEvalBlock) {
        const asift_pair_match p = P.unique[i];
        c += reproj_sq(P.Ht, p.x1, p.y1, p.x2, p.y2) <= th_sq;
    }
    const int t = block_sum(c);
    if (threadIdx.x == 0 && t) atomicAdd(&P.res->r_num, t);
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
ransac_fit_kernel(const EvalProblem *__restrict__ many, const EvalProblem single, const uint32_t *__restrict__ rnd,
                  int n_hyp)
{
    const EvalProblem &P = eprob(many, single, blockIdx.y);
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n_hyp) return;
    const int n = P.res->n_unique;
    double *Hh = P.Hs + 9 * (size_t)h;
    for (int c = 0; c < 9; ++c) Hh[c] = 0.0;
    P.counts[h] = -1;
    if (n < 4) return;
    int idx[4];
    for (int k = 0; k < 4; ++k) idx[k] = (int)(rnd[4 * (size_t)h + k] % (uint32_t)n);
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
            if (idx[a] == idx[b]) return;
    double xs[4], ys[4], us[4], vs[4];
    for (int k = 0; k < 4; ++k) {
        const asift_pair_match p = P.unique[idx[k]];
        xs[k] = p.x1;
        ys[k] = p.y1;
        us[k] = p.x2;
        vs[k] = p.y2;
    }
    double H[9];
    if (!homography4(xs, ys, us, vs, H)) return;
    for (int c = 0; c < 9; ++c) Hh[c] = H[c];
    P.counts[h] = 0;
}

// The threshold test of one pair, decided as reproj_sq(H, ...) <= th_sq is,
// but mostly in fp32: an fp32 evaluation with a rigorous error bound decides
// every pair whose distance is clearly inside or outside the threshold, and
// only pairs within the bound of it take the fp64 path.  With unit roundoff
// u = 2^-24, the rounding of H to fp32 and the products and sums leave |X32 -
// X| <= 4u SX (SX = |h0 x| + |h1 y| + |h2|), likewise for Y and Z; the
// quotient and the difference add a few u more.  The bound below takes 16u
// (four times that) and rejects near-zero denominators, so a decision taken
// in fp32 is the fp64 decision.  The rare undecided case runs out of line,
// so the fp32 loop stays small.
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

// grid (hypothesis groups, CTAs per group, problems)
__global__ void __launch_bounds__(kEvalBlock)
ransac_count_kernel(const EvalProblem *__restrict__ many, const EvalProblem single, int n_hyp, double th_sq)
{
    __shared__ double sH[kHypPerCta][9];
    __shared__ float sHf[kHypPerCta][9];
    __shared__ int sv[kHypPerCta];
    const EvalProblem &P = eprob(many, single, blockIdx.z);
    const int h0 = blockIdx.x * kHypPerCta;
    for (int k = threadIdx.x; k < kHypPerCta * 9; k += blockDim.x) {
        const int h = h0 + k / 9;
        const double hv = h < n_hyp ? P.Hs[9 * (size_t)h + k % 9] : 0.0;
        sH[k / 9][k % 9] = hv;
        sHf[k / 9][k % 9] = (float)hv;
    }
    if (threadIdx.x < kHypPerCta) {
        const int h = h0 + (int)threadIdx.x;
        sv[threadIdx.x] = h < n_hyp && P.counts[h] >= 0;
    }
    __syncthreads();
    const int n = P.res->n_unique;
    // fp32 thresholds strictly inside / outside th_sq by more than their own rounding
    const float th_lo = (float)th_sq * (1.0f - 1e-5f), th_hi = (float)th_sq * (1.0f + 1e-5f);
    int c[kHypPerCta];
#pragma unroll
    for (int k = 0; k < kHypPerCta; ++k) c[k] = 0;
    // the CTAs of one hypothesis group stride over the kept pairs together
    for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) {
        const asift_pair_match p = P.unique[i];
#pragma unroll
        for (int k = 0; k < kHypPerCta; ++k)
            if (sv[k]) c[k] += within_threshold(sH[k], sHf[k], p.x1, p.y1, p.x2, p.y2, th_sq, th_lo, th_hi);
    }
#pragma unroll
    for (int k = 0; k < kHypPerCta; ++k) {
        const int t = block_sum(c[k]);
        if (threadIdx.x == 0 && sv[k] && t) atomicAdd(&P.counts[h0 + k], t);
    }
}

__device__ __forceinline__ bool hyp_better(int c, int h, int bc, int bh) { return c > bc || (c == bc && h < bh); }

// one block per problem
__global__ void __launch_bounds__(kEvalBlock)
ransac_best_kernel(const EvalProblem *__restrict__ many, const EvalProblem single, int n_hyp)
{
    __shared__ int sc[kEvalBlock / 32], sh[kEvalBlock / 32];
    const EvalProblem &P = eprob(many, single, blockIdx.x);
    int bc = -1, bh = n_hyp;
    for (int h = threadIdx.x; h < n_hyp; h += blockDim.x)
        if (P.counts[h] >= 0 && hyp_better(P.counts[h], h, bc, bh)) {
            bc = P.counts[h];
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
        P.res->best_hyp = any ? bh : -1;
        for (int c = 0; c < 9; ++c) P.res->H[c] = any ? P.Hs[9 * (size_t)bh + c] : 0.0;
    }
}

// Over the problem's block range (the whole capacity: the mask beyond the
// kept pairs is cleared).
__global__ void __launch_bounds__(kEvalBlock)
inlier_kernel(const EvalProblem *__restrict__ many, int n_probs, const EvalProblem single)
{
    const EvalProblem &P = eprob(many, single, eval_problem_of_block(many, n_probs, blockIdx.x));
    const asift_eval_result *res = P.res;
    const int n = res->n_unique;
    const bool any = res->best_hyp >= 0;
    const double th_sq = res->ransac_th_sq;
    double H[9];
    for (int c = 0; c < 9; ++c) H[c] = res->H[c];
    const int i = (blockIdx.x - P.blk_off) * kEvalBlock + threadIdx.x;
    bool in = false;
    if (i < n && any) {
        const asift_pair_match p = P.unique[i];
        in = reproj_sq(H, p.x1, p.y1, p.x2, p.y2) <= th_sq;
    }
    if (P.inlier && i < P.cap) P.inlier[i] = (uint8_t)in;
    const int t = block_sum(in);
    if (threadIdx.x == 0 && t) atomicAdd(&P.res->n_inliers, t);
}

// Eq. (1): the scaling coefficient over consecutive pairs of the list (Sec.
// III-A).  Each block sums the terms of its 256 segments in a fixed tree
// order; one block then sums the partials in block order, so the result does
// not depend on scheduling.
__device__ __forceinline__ double block_sum_fixed(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kEvalBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    return sh[0];
}

__global__ void __launch_bounds__(kEvalBlock)
scale_coeff_partial_kernel(const asift_pair_match *__restrict__ pairs, const int32_t *__restrict__ d_n, int cap,
                           double *__restrict__ partials)
{
    __shared__ double sh[kEvalBlock];
    const int n = pair_count(d_n, cap);
    const int i = blockIdx.x * kEvalBlock + threadIdx.x;
    double term = 0.0;
    if (i + 1 < n) {
        const asift_pair_match a = pairs[i], b = pairs[i + 1];
        const double da = hypot((double)b.x1 - (double)a.x1, (double)b.y1 - (double)a.y1);
        const double db = hypot((double)b.x2 - (double)a.x2, (double)b.y2 - (double)a.y2);
        const double w = 1.0 - (double)((int)a.d1 + (int)b.d1) / 1000.0;
        term = (da - db) * w;
    }
    const double t = block_sum_fixed(term, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kEvalBlock)
scale_coeff_final_kernel(const double *__restrict__ partials, int n_part, double *__restrict__ f)
{
    __shared__ double sh[kEvalBlock];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n_part; k += kEvalBlock) acc += partials[k];
    const double t = block_sum_fixed(acc, sh);
    if (threadIdx.x == 0) *f = t;
}

// ---------------------------------------------------------------- host side
static unsigned table_slots(int cap)
{
    unsigned t = 64;
    while (t < 2u * (unsigned)std::max(cap, 1)) t <<= 1;
    return t;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
static int eval_blocks(int cap) { return std::max(1, (cap + kEvalBlock - 1) / kEvalBlock); }

// Scratch of one problem, carved from w (advanced): the duplicate table, the
// keep mask, block counts, the hypotheses' homographies and counts and, with
// own_outputs, the kept pairs, the inlier mask and the result.
static size_t carve_problem(char *&w, bool carve, EvalProblem &P, int cap, int n_hyp, bool own_outputs)
{
    const unsigned slots = table_slots(cap);
    const int blocks = eval_blocks(cap);
    const size_t sizes[8] = {align256(sizeof(int) * slots), align256((size_t)std::max(cap, 1)),
                             align256(sizeof(int32_t) * blocks),
                             align256(sizeof(double) * 9 * (size_t)std::max(n_hyp, 1)),
                             align256(sizeof(int32_t) * (size_t)std::max(n_hyp, 1)),
                             own_outputs ? align256(sizeof(asift_pair_match) * (size_t)std::max(cap, 1)) : 0,
                             own_outputs ? align256((size_t)std::max(cap, 1)) : 0,
                             own_outputs ? align256(sizeof(asift_eval_result)) : 0};
    size_t total = 0;
    for (size_t b : sizes) total += b;
    if (!carve) return total;
    P.cap = cap;
    P.n_blk = blocks;
    P.tmask = slots - 1;
    P.table = reinterpret_cast<int *>(w);
    w += sizes[0];
    P.keep = reinterpret_cast<uint8_t *>(w);
    w += sizes[1];
    P.bcount = reinterpret_cast<int32_t *>(w);
    w += sizes[2];
    P.Hs = reinterpret_cast<double *>(w);
    w += sizes[3];
    P.counts = reinterpret_cast<int32_t *>(w);
    w += sizes[4];
    if (own_outputs) {
        P.unique = reinterpret_cast<asift_pair_match *>(w);
        w += sizes[5];
        P.inlier = reinterpret_cast<uint8_t *>(w);
        w += sizes[6];
        P.res = reinterpret_cast<asift_eval_result *>(w);
        w += sizes[7];
    }
    return total;
}

size_t eval_workspace_bytes(int cap, int n_hyp)
{
    EvalProblem P{};
    char *w = nullptr;
    return carve_problem(w, false, P, cap, n_hyp, false);
}

// The launch sequence for P problems (many: device copy of the list, or
// null with the single problem by value).
static cudaError_t launch_eval_list(const EvalProblem *many, const EvalProblem &single, int P, int total_blk,
                                    int max_blk, int n_hyp, const uint32_t *d_rnd, double th_sq, double ransac_th_sq,
                                    bool any_H, cudaStream_t s)
{
    eval_init_kernel<<<P, 1024, 0, s>>>(many, single, ransac_th_sq);
    dedup_insert_kernel<<<total_blk, kEvalBlock, 0, s>>>(many, P, single);
    dedup_keep_kernel<<<total_blk, kEvalBlock, 0, s>>>(many, P, single);
    block_count_kernel<<<total_blk, kEvalBlock, 0, s>>>(many, P, single);
    compact_kernel<<<total_blk, kEvalBlock, 0, s>>>(many, P, single);
    note_launch(5);
    if (any_H) {
        precision_kernel<<<total_blk, kEvalBlock, 0, s>>>(many, P, single, th_sq);
        note_launch();
    }
    if (n_hyp > 0) {
        ransac_fit_kernel<<<dim3((n_hyp + 31) / 32, P), 32, 0, s>>>(many, single, d_rnd, n_hyp);
        // hypothesis groups x CTAs per group x problems: about two CTAs per
        // SM, no more CTAs per group than a problem's blocks of pairs
        const int hyp_blocks = (n_hyp + kHypPerCta - 1) / kHypPerCta;
        const long long per = (long long)hyp_blocks * P;
        const int gy = (int)std::max(1LL, std::min((2LL * 152 + per - 1) / per, (long long)max_blk));
        ransac_count_kernel<<<dim3(hyp_blocks, gy, P), kEvalBlock, 0, s>>>(many, single, n_hyp, ransac_th_sq);
        ransac_best_kernel<<<P, kEvalBlock, 0, s>>>(many, single, n_hyp);
        note_launch(3);
    }
    inlier_kernel<<<total_blk, kEvalBlock, 0, s>>>(many, P, single);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_eval(const asift_pair_match *d_pairs, const int32_t *d_n, int cap, const double *h_H_true,
                        double th_sq, const uint32_t *d_rnd, int n_hyp, double ransac_th_sq,
                        asift_pair_match *d_unique, uint8_t *d_inlier, int32_t *d_hyp_counts,
                        asift_eval_result *d_res, void *d_ws, cudaStream_t s)
{
    EvalProblem P{};
    char *w = static_cast<char *>(d_ws);
    carve_problem(w, true, P, cap, n_hyp, false);
    P.pairs = d_pairs;
    P.d_n = d_n;
    P.blk_off = 0;
    P.unique = d_unique;
    P.inlier = d_inlier;
    P.res = d_res;
    if (d_hyp_counts) P.counts = d_hyp_counts;
    P.has_H = h_H_true != nullptr;
    for (int c = 0; c < 9; ++c) P.Ht[c] = h_H_true ? h_H_true[c] : 0.0;
    return launch_eval_list(nullptr, P, 1, P.n_blk, P.n_blk, n_hyp, d_rnd, th_sq, ransac_th_sq, P.has_H, s);
}

size_t scale_coeff_workspace_bytes(int cap) { return sizeof(double) * (size_t)eval_blocks(cap); }

cudaError_t launch_scale_coeff(const asift_pair_match *d_pairs, const int32_t *d_n, int cap, double *d_f, void *d_ws,
                               cudaStream_t s)
{
    const int blocks = eval_blocks(cap);
    double *partials = static_cast<double *>(d_ws);
    scale_coeff_partial_kernel<<<blocks, kEvalBlock, 0, s>>>(d_pairs, d_n, cap, partials);
    scale_coeff_final_kernel<<<1, kEvalBlock, 0, s>>>(partials, blocks, d_f);
    note_launch(2);
    return cudaGetLastError();
}

// ---- batched form: the pairs of a plan, one launch per stage
size_t eval_batch_workspace_bytes(const int *caps, int n, int n_hyp)
{
    size_t b = align256(sizeof(EvalProblem) * (size_t)std::max(n, 1));
    EvalProblem P{};
    char *w = nullptr;
    for (int i = 0; i < n; ++i) b += carve_problem(w, false, P, caps[i], n_hyp, true);
    return b;
}

static void carve_batch(void *d_ws, const int *caps, int n, int n_hyp, std::vector<EvalProblem> &probs)
{
    probs.assign(n, EvalProblem{});
    char *w = static_cast<char *>(d_ws) + align256(sizeof(EvalProblem) * (size_t)std::max(n, 1));
    int off = 0;
    for (int i = 0; i < n; ++i) {
        carve_problem(w, true, probs[i], caps[i], n_hyp, true);
        probs[i].blk_off = off;
        off += probs[i].n_blk;
    }
}

void eval_batch_outputs(void *d_ws, const int *caps, int n, int n_hyp, int i, asift_pair_match **unique,
                        uint8_t **inlier, int32_t **counts, asift_eval_result **res)
{
    std::vector<EvalProblem> probs;
    carve_batch(d_ws, caps, n, n_hyp, probs);
    if (unique) *unique = probs[i].unique;
    if (inlier) *inlier = probs[i].inlier;
    if (counts) *counts = probs[i].counts;
    if (res) *res = probs[i].res;
}

cudaError_t launch_eval_batch(asift_pair_match *const *pairs, int32_t *d_ns, const int *caps, int n,
                              const double *h_H_true, double th_sq, const uint32_t *d_rnd, int n_hyp,
                              double ransac_th_sq, void *d_ws, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    std::vector<EvalProblem> probs;
    carve_batch(d_ws, caps, n, n_hyp, probs);
    int total = 0, max_blk = 1;
    for (int i = 0; i < n; ++i) {
        EvalProblem &P = probs[i];
        P.pairs = pairs[i];
        P.d_n = d_ns + i;
        P.has_H = h_H_true != nullptr;
        for (int c = 0; c < 9; ++c) P.Ht[c] = h_H_true ? h_H_true[9 * (size_t)i + c] : 0.0;
        total += P.n_blk;
        max_blk = std::max(max_blk, P.n_blk);
    }
    EvalProblem *d_probs = static_cast<EvalProblem *>(d_ws);
    // pageable source: the copy is staged before the call returns
    const cudaError_t e = cudaMemcpyAsync(d_probs, probs.data(), sizeof(EvalProblem) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return launch_eval_list(d_probs, probs[0], n, total, max_blk, n_hyp, d_rnd, th_sq, ransac_th_sq,
                            h_H_true != nullptr, s);
}

}  // namespace asift
