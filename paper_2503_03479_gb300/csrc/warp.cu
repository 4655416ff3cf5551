// warp.cu -- affine view simulation (Eq. (2)-(4)) on sm_103a.
//
// One CTA produces a kWarpTW x kWarpTH tile of one view.  A view row j only
// depends on canvas row j (the tilt acts along canvas x), so the tile needs a
// canvas strip of kWarpTH rows and about t*kWarpTW + 2K + 6 columns.  The CTA:
//   1. computes the rotated canvas C on that strip into shared memory
//      (normalised 6x6 Lanczos-3, Eq. (3)-(4); geometry in exact Q32);
//   2. blurs the strip along x with the Gaussian taps into shared memory (B);
//   3. resamples B at X = t (x' - (Wv-1)/2) + (Wr-1)/2 with Lanczos-3 and
//      writes fp32 (optional), rint-to-u8 and the footprint mask.
// Every launch covers a list of views (one view for the per-view form, all
// views of several images for the batched form); a CTA finds its view by a
// binary search over the views' first tile index.
#include "common.cuh"
#include "kernels.h"

namespace asift {

// Normalised Lanczos-3 weights (Eq. (4), a = 3) of the taps floor(p) + m,
// m = -2..3, at fractional position f in [0, 1) given as Q32 bits `lo`.
// L(f - m) = 3 sin(pi (f - m)) sin(pi (f - m)/3) / (pi (f - m))^2 and
// sin(pi (f - m)) = (-1)^m sin(pi f): the common factor 3 sin(pi f)/pi^2
// cancels in the normalisation, leaving
//   w_m  ~  (-1)^m sin(pi f/3 - pi m/3) / (f - m)^2,
// whose six sines follow from one sincospi(f/3) by angle addition.  f = 0
// (lo == 0) is the identity.
__device__ __forceinline__ void lanczos3_weights(uint32_t lo, float w[6])
{
    if (lo == 0u) {
        w[0] = w[1] = w[3] = w[4] = w[5] = 0.f;
        w[2] = 1.f;
        return;
    }
    const float f = __uint2float_rz(lo) * 2.3283064365386963e-10f;   // < 1
    float s, c;
    sincospif(f * (1.0f / 3.0f), &s, &c);
    const float hs = 0.5f * s, hc = 0.86602540378443864676f * c;
    float n0 = hc - hs, n1 = -(hs + hc), n2 = s, n3 = hc - hs, n4 = -(hs + hc), n5 = s;
    float d0 = f + 2.f, d1 = f + 1.f, d2 = f, d3 = f - 1.f, d4 = f - 2.f, d5 = f - 3.f;
    n0 = __fdiv_rn(n0, d0 * d0);
    n1 = __fdiv_rn(n1, d1 * d1);
    n2 = __fdiv_rn(n2, d2 * d2);
    n3 = __fdiv_rn(n3, d3 * d3);
    n4 = __fdiv_rn(n4, d4 * d4);
    n5 = __fdiv_rn(n5, d5 * d5);
    const float inv = __frcp_rn(((n0 + n1) + (n2 + n3)) + (n4 + n5));
    w[0] = n0 * inv; w[1] = n1 * inv; w[2] = n2 * inv;
    w[3] = n3 * inv; w[4] = n4 * inv; w[5] = n5 * inv;
}

__global__ void u8_to_f32_kernel(const uint8_t *__restrict__ src, int pitch, int W, int H,
                                 float *__restrict__ dst)
{
    const long long n = (long long)W * H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (long long)y * W);
        dst[i] = (float)src[(size_t)y * pitch + x];
    }
}

__global__ void __launch_bounds__(kWarpThreads)
warp_view_kernel(const DevView *__restrict__ views, int n_views, int cw_max, int bw_max,
                 uint8_t *__restrict__ out_u8, uint8_t *__restrict__ out_mask, float *__restrict__ out_f32)
{
    extern __shared__ float smem[];
    float *Cs = smem;                              // [kWarpTH][cw_max]
    float *Bs = smem + kWarpTH * cw_max;           // [kWarpTH][bw_max]
    __shared__ float gs[ASIFT_MAX_GAUSS];

    const int tile = blockIdx.x;
    const int vi = find_owner(views, n_views, tile, [](const DevView &v) { return v.tile_start; });
    const DevView &V = views[vi];
    const int lt = tile - V.tile_start;
    const int ty = lt / V.ntx, tx = lt - ty * V.ntx;
    const int xa = tx * kWarpTW, xb = min(xa + kWarpTW, V.Wv) - 1;
    const int j0 = ty * kWarpTH, j1 = min(j0 + kWarpTH, V.Hv) - 1;
    const int nrows = j1 - j0 + 1;
    const int Wr = V.Wr, K = V.K;
    const long long HALF = 2147483648LL;
    const long long xoff = (long long)(Wr - 1) * HALF;

    const long long Xa = V.tq * (2LL * xa - V.Wv + 1) + xoff;
    const long long Xb = V.tq * (2LL * xb - V.Wv + 1) + xoff;
    const int bx0 = max(0, (int)(Xa >> 32) - 2), bx1 = min(Wr - 1, (int)(Xb >> 32) + 3);
    const int cx0 = max(0, bx0 - K), cx1 = min(Wr - 1, bx1 + K);
    const int cw = cx1 - cx0 + 1, bw = bx1 - bx0 + 1;

    for (int k = threadIdx.x; k <= K; k += blockDim.x) gs[k] = V.g[k];

    // 1. rotated canvas strip (Eq. (3)-(4))
    const float *__restrict__ src = V.src;
    const int sp = V.src_pitch, W = V.W, H = V.H;
    const long long xlim = (long long)(2 * W - 1) * HALF, ylim = (long long)(2 * H - 1) * HALF;
    for (int e = threadIdx.x; e < nrows * cw; e += blockDim.x) {
        const int r = e / cw, c = e - r * cw;
        const int i = cx0 + c, j = j0 + r;
        const long long dx2 = 2LL * i - Wr + 1, dy2 = 2LL * j - V.Hr + 1;
        const long long px = V.cq * dx2 + V.sq * dy2 + (long long)(W - 1) * HALF;
        const long long py = -V.sq * dx2 + V.cq * dy2 + (long long)(H - 1) * HALF;
        float acc = 0.f;
        if (px >= -HALF && px < xlim && py >= -HALF && py < ylim) {
            float wx[6], wy[6];
            lanczos3_weights((uint32_t)px, wx);
            lanczos3_weights((uint32_t)py, wy);
            const int x0 = (int)(px >> 32), y0 = (int)(py >> 32);
            int xs[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) xs[m] = clampi(x0 + m - 2, 0, W - 1);
#pragma unroll
            for (int n = 0; n < 6; ++n) {
                const float *row = src + (size_t)clampi(y0 + n - 2, 0, H - 1) * sp;
                float a = 0.f;
#pragma unroll
                for (int m = 0; m < 6; ++m) a = fmaf(wx[m], __ldg(row + xs[m]), a);
                acc = fmaf(wy[n], a, acc);
            }
        }
        Cs[r * cw_max + c] = acc;
    }
    __syncthreads();

    // 2. Gaussian along canvas x (clamped to the canvas)
    for (int e = threadIdx.x; e < nrows * bw; e += blockDim.x) {
        const int r = e / bw, c = e - r * bw;
        const int i = bx0 + c;
        const float *Crow = Cs + r * cw_max - cx0;
        float acc = gs[0] * Crow[i];
        for (int k = 1; k <= K; ++k)
            acc = fmaf(gs[k], Crow[clampi(i - k, 0, Wr - 1)] + Crow[clampi(i + k, 0, Wr - 1)], acc);
        Bs[r * bw_max + c] = acc;
    }
    __syncthreads();

    // 3. tilt resampling, quantisation and the footprint mask
    const int ncols = xb - xa + 1;
    const long long mxlo = HALF, mxhi = (long long)(2 * W - 3) * HALF;
    const long long mylo = HALF, myhi = (long long)(2 * H - 3) * HALF;
    for (int e = threadIdx.x; e < nrows * ncols; e += blockDim.x) {
        const int r = e / ncols, c = e - r * ncols;
        const int x = xa + c, j = j0 + r;
        const long long X = V.tq * (2LL * x - V.Wv + 1) + xoff;
        const int x0 = (int)(X >> 32);
        float w[6];
        lanczos3_weights((uint32_t)X, w);
        const float *Brow = Bs + r * bw_max - bx0;
        float v = 0.f;
#pragma unroll
        for (int m = 0; m < 6; ++m) v = fmaf(w[m], Brow[clampi(x0 + m - 2, 0, Wr - 1)], v);
        int valid = 1;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = x0 + q;
            if (i < 0 || i >= Wr) { valid = 0; continue; }
            const long long dx2 = 2LL * i - Wr + 1, dy2 = 2LL * j - V.Hr + 1;
            const long long px = V.cq * dx2 + V.sq * dy2 + (long long)(W - 1) * HALF;
            const long long py = -V.sq * dx2 + V.cq * dy2 + (long long)(H - 1) * HALF;
            valid &= (px >= mxlo && px <= mxhi && py >= mylo && py <= myhi);
        }
        const size_t o = (size_t)V.out_off + (size_t)j * V.Wv + x;
        if (out_f32) out_f32[o] = v;
        const int q8 = __float2int_rn(v);
        out_u8[o] = (uint8_t)min(255, max(0, q8));
        out_mask[o] = (uint8_t)valid;
    }
}

// ---------------------------------------------------------------- host side
void warp_strip_widths(const asift_view_desc &v, int *cw, int *bw)
{
    // columns of B a tile needs: floor(X) - 2 .. floor(X) + 3 over kWarpTW view
    // columns spaced t apart, plus the Gaussian reach K on both sides for C.
    const int span = (int)std::ceil(v.t * (kWarpTW - 1)) + 1;
    *bw = span + 6 + 1;
    *cw = *bw + 2 * v.K;
}

cudaError_t launch_u8_to_f32(const uint8_t *src, int pitch, int W, int H, float *dst, cudaStream_t s)
{
    const long long n = (long long)W * H;
    int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
    u8_to_f32_kernel<<<blocks, 256, 0, s>>>(src, pitch, W, H, dst);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_warp(const DevView *d_views, int n_views, int n_tiles, int cw_max, int bw_max,
                        uint8_t *u8, uint8_t *mask, float *f32, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * (size_t)kWarpTH * (cw_max + bw_max);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(warp_view_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    warp_view_kernel<<<n_tiles, kWarpThreads, smem, s>>>(d_views, n_views, cw_max, bw_max, u8, mask, f32);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asift
