// sift_match.cu -- brute-force L2 matching of SIFT descriptors with the ratio
// test, the matching of the precise stage (Sec. III-C) and the input of the
// base-image selection of Eq. (1) (Sec. III-A), on sm_103a.
//
// Distances are decided in fp32 in one fixed order, so that the argmax is the
// same on every implementation that keeps it: the squared distance of query i
// and train j is the fp32 sum over c = 0, 1, ..., 127 in that order of e_c^2
// (e_c = q_c - t_c rounded to fp32), each term added by one fused
// multiply-add.  The kernel tiles 64 queries x 64 trains per step; each
// thread owns a 4 x 4 block of (query, train) accumulators and walks c in
// order, so every pair's sum is that chain.  Distances are non-negative, so
// their fp32 bits order like the values: a key (bits << 32 | train index)
// ordered as an integer gives the smallest distance, then the lowest index,
// and the running nearest and second-nearest are a min / max network on keys
// (the second equals the first on a tie).  Train slices write partial keys
// that a merge kernel combines; a single-block scan writes the accepted pairs
// in query order.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace asift {

constexpr int kSmT = 64;                 // queries / trains per tile
constexpr int kSmThreads = 256;          // 16 x 16 threads, 4 x 4 pairs each
constexpr int kSmPitch = kSmT + 4;       // transposed tile row pitch (floats)
constexpr int kSmMaxSlices = 32;
constexpr unsigned long long kSmNoKey = ~0ull;

__device__ __forceinline__ int sm_count(const int32_t *d, int cap) { return d ? min(max(*d, 0), cap) : cap; }

__device__ __forceinline__ void sm_insert(unsigned long long key, unsigned long long &b1, unsigned long long &b2)
{
    b2 = min(b2, max(b1, key));
    b1 = min(b1, key);
}

// Stages rows [r0, r0 + kSmT) of a (rows x 128) descriptor array transposed:
// S[c][r] (rows past n read as zeros).
__device__ __forceinline__ void stage_tile(float *S, const float *__restrict__ src, int r0, int n)
{
    for (int el = threadIdx.x; el < kSmT * 32; el += kSmThreads) {
        const int r = el & (kSmT - 1), c4 = el / kSmT;   // a warp: 32 rows, one float4 column (distinct banks)
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r0 + r < n) v = __ldg(reinterpret_cast<const float4 *>(src + (size_t)(r0 + r) * 128) + c4);
        S[(4 * c4 + 0) * kSmPitch + r] = v.x;
        S[(4 * c4 + 1) * kSmPitch + r] = v.y;
        S[(4 * c4 + 2) * kSmPitch + r] = v.z;
        S[(4 * c4 + 3) * kSmPitch + r] = v.w;
    }
}

// grid (query blocks of 64, train slices): partial keys of slice s at
// part[(s * nq_cap + i) * 2 + {0, 1}].
__global__ void __launch_bounds__(kSmThreads)
sift_l2_kernel(const float *__restrict__ q, const int32_t *__restrict__ d_nq, int nq_cap, const float *__restrict__ t,
               const int32_t *__restrict__ d_nt, int nt_cap, int n_slices, unsigned long long *__restrict__ part)
{
    extern __shared__ float4 sm4[];
    float *Qs = reinterpret_cast<float *>(sm4);          // [128][kSmPitch]
    float *Ts = Qs + 128 * kSmPitch;
    const int nq = sm_count(d_nq, nq_cap), nt = sm_count(d_nt, nt_cap);
    const int q0 = blockIdx.x * kSmT;
    if (q0 >= nq) return;
    // this slice's trains: whole tiles, split evenly over the slices
    const int tiles = (nt + kSmT - 1) / kSmT;
    const int s = blockIdx.y;
    const int tb = (int)((long long)tiles * s / n_slices), te = (int)((long long)tiles * (s + 1) / n_slices);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    unsigned long long b1[4], b2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) b1[i] = b2[i] = kSmNoKey;
    stage_tile(Qs, q, q0, nq);
    for (int tt = tb; tt < te; ++tt) {
        const int t0 = tt * kSmT;
        __syncthreads();                                 // everyone is done with the previous train tile
        stage_tile(Ts, t, t0, nt);
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
        for (int c = 0; c < 128; ++c) {
            const float4 a = *reinterpret_cast<const float4 *>(Qs + c * kSmPitch + 4 * ty);
            const float4 b = *reinterpret_cast<const float4 *>(Ts + c * kSmPitch + 4 * tx);
            const float qa[4] = {a.x, a.y, a.z, a.w}, tb4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float e = __fsub_rn(qa[i], tb4[j]);
                    acc[i][j] = __fmaf_rn(e, e, acc[i][j]);
                }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int tj = t0 + 4 * tx + j;
            if (tj < nt) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    sm_insert(((unsigned long long)__float_as_uint(acc[i][j]) << 32) | (unsigned)tj, b1[i], b2[i]);
            }
        }
    }
    // the 16 threads of a row (lanes with the same lane >> 4) combine their keys
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const unsigned long long o1 = __shfl_xor_sync(0xffffffffu, b1[i], o);
            const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, b2[i], o);
            sm_insert(o1, b1[i], b2[i]);
            sm_insert(o2, b1[i], b2[i]);
        }
    }
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int qi = q0 + 4 * ty + i;
            if (qi < nq) {
                part[((size_t)s * nq_cap + qi) * 2] = b1[i];
                part[((size_t)s * nq_cap + qi) * 2 + 1] = b2[i];
            }
        }
    }
}

// One thread per query: the slices' keys -> nearest, second nearest, ratio test.
__global__ void __launch_bounds__(256)
sift_l2_merge_kernel(const unsigned long long *__restrict__ part, int n_slices, const int32_t *__restrict__ d_nq,
                     int nq_cap, const int32_t *__restrict__ d_nt, int nt_cap, float r2, asift_l2_match *__restrict__ out,
                     uint8_t *__restrict__ accept)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nq = sm_count(d_nq, nq_cap), nt = sm_count(d_nt, nt_cap);
    if (i >= nq) return;
    unsigned long long b1 = kSmNoKey, b2 = kSmNoKey;
    if (nt > 0)
        for (int s = 0; s < n_slices; ++s) {
            sm_insert(part[((size_t)s * nq_cap + i) * 2], b1, b2);
            sm_insert(part[((size_t)s * nq_cap + i) * 2 + 1], b1, b2);
        }
    asift_l2_match m;
    m.best = b1 == kSmNoKey ? -1 : (int32_t)(b1 & 0xffffffffu);
    m.d1 = b1 == kSmNoKey ? __int_as_float(0x7f800000) : __uint_as_float((unsigned)(b1 >> 32));
    m.d2 = b2 == kSmNoKey ? __int_as_float(0x7f800000) : __uint_as_float((unsigned)(b2 >> 32));
    out[i] = m;
    accept[i] = (uint8_t)(m.best >= 0 && nt >= 2 && m.d1 < __fmul_rn(r2, m.d2));
}

// The descriptor distance of a pair for Eq. (1): the L2 distance at the
// conventional scale of integer SIFT descriptors (norm 512), rounded.
__device__ __forceinline__ uint16_t des512(float dsq)
{
    const float d = 512.0f * sqrtf(fmaxf(dsq, 0.0f));
    return (uint16_t)min(65535, __float2int_rn(d));
}

// One block: the accepted queries in query order -> asift_pair_match.
__global__ void __launch_bounds__(1024)
sift_pairs_kernel(const asift_l2_match *__restrict__ m, const uint8_t *__restrict__ accept, const int32_t *__restrict__ d_nq,
                  int nq_cap, const asift_sift_kp *__restrict__ kq, const asift_sift_kp *__restrict__ kt,
                  asift_pair_match *__restrict__ pairs, int cap, int32_t *__restrict__ d_n, int32_t *__restrict__ status)
{
    __shared__ int wsum[32];
    __shared__ int base, chunk;
    const int nq = sm_count(d_nq, nq_cap);
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int q0 = 0; q0 < nq; q0 += 1024) {
        const int i = q0 + (int)threadIdx.x;
        const bool a = i < nq && accept[i];
        const unsigned bal = __ballot_sync(0xffffffffu, a);
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {                      // exclusive prefix of the warps' counts
            int acc = 0;
            for (int k = 0; k < 32; ++k) { const int v = wsum[k]; wsum[k] = acc; acc += v; }
            chunk = acc;
        }
        __syncthreads();
        if (a) {
            const int o = base + wsum[w] + __popc(bal & ((1u << lane) - 1u));
            if (o < cap) {
                const asift_l2_match mm = m[i];
                asift_pair_match p;
                p.x1 = kq[i].x;
                p.y1 = kq[i].y;
                p.x2 = kt[mm.best].x;
                p.y2 = kt[mm.best].y;
                p.q = i;
                p.t = mm.best;
                p.d1 = des512(mm.d1);
                p.d2 = des512(mm.d2);
                pairs[o] = p;
            }
        }
        __syncthreads();                             // everyone has read base and wsum
        if (threadIdx.x == 0) base += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *d_n = base;
        if (base > cap) set_status(status, ASIFT_ERR_CAPACITY);
    }
}

// ---------------------------------------------------------------- host side
int sift_match_slices(int nq, int nt)
{
    const int qb = std::max(1, (nq + kSmT - 1) / kSmT), tt = std::max(1, (nt + kSmT - 1) / kSmT);
    const int want = (2 * device_sm_count() + qb - 1) / qb;   // about two CTAs per SM
    return std::max(1, std::min({want, tt, kSmMaxSlices}));
}

size_t sift_match_workspace_bytes(int nq, int nt)
{
    return 256 + (size_t)kSmMaxSlices * std::max(nq, 1) * 2 * sizeof(unsigned long long) + 256 +
           (size_t)std::max(nq, 1) + 256;
}

cudaError_t launch_sift_match(const float *q, int nq, const int32_t *d_nq, const float *t, int nt, const int32_t *d_nt,
                              double ratio, const asift_sift_kp *kq, const asift_sift_kp *kt, asift_l2_match *out,
                              asift_pair_match *pairs, int cap, int32_t *d_n, void *ws, cudaStream_t s)
{
    char *w = static_cast<char *>(ws);
    int32_t *status = reinterpret_cast<int32_t *>(w);
    unsigned long long *part = reinterpret_cast<unsigned long long *>(w + 256);
    uint8_t *accept = reinterpret_cast<uint8_t *>(w + 256 + (size_t)kSmMaxSlices * std::max(nq, 1) * 16 + 256);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (nq > 0) {
        const int ns = sift_match_slices(nq, nt);
        if (nt > 0) {
            const size_t smem = 2 * 128 * kSmPitch * sizeof(float);
            e = ensure_dynamic_smem((const void *)sift_l2_kernel, smem);
            if (e != cudaSuccess) return e;
            sift_l2_kernel<<<dim3((nq + kSmT - 1) / kSmT, ns), kSmThreads, smem, s>>>(q, d_nq, nq, t, d_nt, nt, ns,
                                                                                      part);
            note_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        sift_l2_merge_kernel<<<(nq + 255) / 256, 256, 0, s>>>(part, nt > 0 ? ns : 0, d_nq, nq, d_nt, nt,
                                                              (float)(ratio * ratio), out, accept);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (d_n) {
        if (nq > 0 && kq && kt) {
            sift_pairs_kernel<<<1, 1024, 0, s>>>(out, accept, d_nq, nq, kq, kt, pairs, cap, d_n, status);
            note_launch();
            e = cudaGetLastError();
        } else {
            e = cudaMemsetAsync(d_n, 0, sizeof(int32_t), s);
        }
    }
    return e;
}

}  // namespace asift
