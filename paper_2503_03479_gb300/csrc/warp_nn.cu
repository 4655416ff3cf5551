// warp_nn.cu -- nearest-neighbour affine views (the coarse stage's
// interpolation, Sec. III-B) on sm_103a.  Same tiles, view descriptors,
// outputs and mask as warp_view_kernel (warp.cu); only the two resamplings
// differ: the canvas takes the source pixel nearest to each canvas pixel's
// source point and a view column takes the blurred canvas column nearest to
// its position X.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace asift {

namespace {
struct NNGeom {               // Q32 map of canvas (i, j) to the source point, Eq. (2) with the scale in (cq, sq)
    long long cq, sq, ox, oy;
    int Wr, Hr;
    __device__ __forceinline__ void map(int i, int j, long long &px, long long &py) const
    {
        const long long dx2 = 2LL * i - Wr + 1, dy2 = 2LL * j - Hr + 1;
        px = cq * dx2 + sq * dy2 + ox;
        py = -sq * dx2 + cq * dy2 + oy;
    }
};
}  // namespace

// ---------------------------------------------------------------- nearest-neighbour views
// The coarse stage's interpolation (Sec. III-B): the canvas takes the source
// pixel nearest to each canvas pixel's source point, round(p) = floor(p + 1/2)
// in Q32 (0 outside [-0.5, W-0.5) x [-0.5, H-0.5)); the Gaussian along x is
// unchanged; view column x' takes the blurred canvas column nearest to X,
// clamped to the canvas.  Same tiles, outputs and mask as warp_view_kernel.
//   1. the canvas strip of the tile's rows over the columns the nearest
//      columns' Gaussian windows reach (clamped to the canvas): every thread
//      walks 4 rows of one column, stepping the Q32 source point by one row;
//   2. each view pixel sums the 2K+1 Gaussian taps around its nearest column.
constexpr int kNNRowsPerThread = 4;

__device__ __forceinline__ void warp_nn_tile(int tile, const DevView *__restrict__ views, int n_views, int cwp,
                                             uint8_t *__restrict__ out_u8, uint8_t *__restrict__ out_mask,
                                             float *__restrict__ out_f32)
{
    extern __shared__ float4 smem4[];
    float *Cs = reinterpret_cast<float *>(smem4);      // [kWarpTH][cwp]
    float *gs = Cs + kWarpTH * cwp;                    // Gaussian taps g_0 .. g_K

    const int vi = find_owner(views, n_views, tile, [](const DevView &v) { return v.tile_start; });
    const DevView &V = views[vi];
    const int lt = tile - V.tile_start;
    const int ty = lt / V.ntx, tx = lt - ty * V.ntx;
    const int xa = tx * V.tw, xb = min(xa + V.tw, V.Wv) - 1;
    const int j0 = ty * kWarpTH, j1 = min(j0 + kWarpTH, V.Hv) - 1;
    const int nrows = j1 - j0 + 1;
    const int Wr = V.Wr, K = V.K, W = V.W, H = V.H;
    const long long HALF = 2147483648LL;
    const long long xoff = (long long)(Wr - 1) * HALF;
    const NNGeom G{V.cq, V.sq, (long long)(W - 1) * HALF, (long long)(H - 1) * HALF, Wr, V.Hr};

    const long long Xa = V.tq * (2LL * xa - V.Wv + 1) + xoff;
    const long long Xb = V.tq * (2LL * xb - V.Wv + 1) + xoff;
    const int na = clampi((int)((Xa + HALF) >> 32), 0, Wr - 1), nb = clampi((int)((Xb + HALF) >> 32), 0, Wr - 1);
    const int lo = max(0, na - K);
    const int cw = min(min(Wr - 1, nb + K) - lo + 1, cwp);     // never above cwp: see warp_nn_strip_fits

    for (int k = threadIdx.x; k <= K; k += blockDim.x) gs[k] = V.g[k];

    // 1. canvas strip
    {
        const int rg = (int)(threadIdx.x / 64u) * kNNRowsPerThread;
        const long long xlim = (long long)(2 * W - 1) * HALF, ylim = (long long)(2 * H - 1) * HALF;
        const long long dpx = 2LL * V.sq, dpy = 2LL * V.cq;
        const float *__restrict__ src = V.src;
        const int sp = V.src_pitch;
        for (int c = (int)(threadIdx.x & 63u); c < cw; c += 64) {
            long long px, py;
            G.map(lo + c, j0 + rg, px, py);
#pragma unroll
            for (int q = 0; q < kNNRowsPerThread; ++q, px += dpx, py += dpy) {
                const int r = rg + q;
                if (r >= nrows) break;
                float val = 0.f;
                if (px >= -HALF && px < xlim && py >= -HALF && py < ylim)
                    val = __ldg(src + (size_t)((py + HALF) >> 32) * sp + (int)((px + HALF) >> 32));
                Cs[r * cwp + c] = val;
            }
        }
    }
    __syncthreads();

    // 2. Gaussian at the nearest column, quantisation and the footprint mask
    {
        const int c = (int)(threadIdx.x & 63u), rg = (int)(threadIdx.x / 64u);
        const int ncols = xb - xa + 1;
        constexpr int kRowStep = kWarpThreads / 64;
        if (c < ncols) {
            const int x = xa + c;
            const long long X = V.tq * (2LL * x - V.Wv + 1) + xoff;
            const int xn = clampi((int)((X + HALF) >> 32), 0, Wr - 1);
            const int x0 = (int)(X >> 32);
            float acc[kWarpTH / kRowStep];
#pragma unroll
            for (int q = 0; q < kWarpTH / kRowStep; ++q) acc[q] = 0.f;
            const float *Cb = Cs + rg * cwp;
            if (xn - K >= 0 && xn + K <= Wr - 1) {
                const float *b = Cb + (xn - lo);
                for (int k = -K; k <= K; ++k) {
                    const float g = gs[abs(k)];
#pragma unroll
                    for (int q = 0; q < kWarpTH / kRowStep; ++q) acc[q] = fmaf(g, b[q * kRowStep * cwp - k], acc[q]);
                }
            } else {
                for (int k = -K; k <= K; ++k) {
                    const float g = gs[abs(k)];
                    const int i = clampi(xn - k, 0, Wr - 1) - lo;
#pragma unroll
                    for (int q = 0; q < kWarpTH / kRowStep; ++q) acc[q] = fmaf(g, Cb[q * kRowStep * cwp + i], acc[q]);
                }
            }
            const long long mxlo = HALF, mxhi = (long long)(2 * W - 3) * HALF;
            const long long mylo = HALF, myhi = (long long)(2 * H - 3) * HALF;
            const long long dpx = 2LL * kRowStep * V.sq, dpy = 2LL * kRowStep * V.cq;
            const bool cols_ok = x0 >= 0 && x0 + 1 <= Wr - 1;
            long long pxa, pya, pxb, pyb;
            G.map(clampi(x0, 0, Wr - 1), j0 + rg, pxa, pya);
            G.map(clampi(x0 + 1, 0, Wr - 1), j0 + rg, pxb, pyb);
#pragma unroll
            for (int q = 0; q < kWarpTH / kRowStep; ++q, pxa += dpx, pya += dpy, pxb += dpx, pyb += dpy) {
                const int r = rg + q * kRowStep;
                if (r >= nrows) break;
                const int j = j0 + r;
                const bool valid = cols_ok && pxa >= mxlo && pxa <= mxhi && pya >= mylo && pya <= myhi &&
                                   pxb >= mxlo && pxb <= mxhi && pyb >= mylo && pyb <= myhi;
                const size_t o = (size_t)V.out_off + (size_t)j * V.Wv + x;
                if (out_f32) out_f32[o] = acc[q];
                out_u8[o] = (uint8_t)min(255, max(0, __float2int_rn(acc[q])));
                out_mask[o] = (uint8_t)valid;
            }
        }
    }
}

__global__ void __launch_bounds__(kWarpThreads)
warp_nn_kernel(int n_tiles, const DevView *__restrict__ views, int n_views, int cwp, uint8_t *__restrict__ out_u8,
               uint8_t *__restrict__ out_mask, float *__restrict__ out_f32)
{
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        warp_nn_tile(tile, views, n_views, cwp, out_u8, out_mask, out_f32);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side
// Strip width of the nearest-neighbour form for a tile of tw view columns:
// the nearest columns of the tile's first and last view columns lie at most
// t (tw - 1) + 1 (+ the Q31 rounding of t) apart, plus K on both sides; within
// the Lanczos strip width of warp_strip_widths for the same tw.
int warp_nn_strip_width(const asift_view_desc &v, int tw) { return (int)std::ceil(v.t * (tw - 1)) + 2 + 2 * v.K; }

cudaError_t launch_warp_nn(const DevView *d_views, int n_views, int n_tiles, int cw_max, uint8_t *u8, uint8_t *mask,
                           float *f32, cudaStream_t s, int grid)
{
    if (n_tiles <= 0) return cudaSuccess;
    const int cwp = cw_max | 1;                          // odd pitch
    const size_t smem = sizeof(float) * ((size_t)kWarpTH * cwp + ASIFT_MAX_GAUSS);
    const cudaError_t e = ensure_dynamic_smem((const void *)warp_nn_kernel, smem);
    if (e != cudaSuccess) return e;
    const int g = (grid > 0 && grid < n_tiles) ? grid : n_tiles;
    warp_nn_kernel<<<g, kWarpThreads, smem, s>>>(n_tiles, d_views, n_views, cwp, u8, mask, f32);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asift
