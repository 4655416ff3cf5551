// warp_precise.cu -- Lanczos-a affine views (Eq. (2)-(4) with a general a) on
// sm_103a, for the precise stage's reproduction of the best view (Sec. III-C:
// a = 4, an 8 x 8 window).  One view per pair is reproduced, so this kernel
// favours a plain structure over the staged pipeline of warp.cu; it also
// serves a = 3 as an independent check of that kernel.
//
// Same tiles, view descriptors, outputs and mask as warp_view_kernel.  Per
// tile (tw view columns x 16 rows) the CTA computes
//   1. the canvas strip C over the columns the tile's Gaussian windows reach
//      (clamped to the canvas): 2a x 2a normalised Lanczos-a taps of the fp32
//      source through the L1 cache, clamp-to-edge, 0 outside the footprint;
//   2. B = the Gaussian along x at the canvas columns the tilt taps read;
//   3. the 2a-tap Lanczos-a tilt at X = t (x' - (Wv-1)/2) + (Wr-1)/2.
// Positions are the Q32 fixed point of the main path; weights are fp32
// (sinpi-based), normalised to sum 1.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace asift {

namespace {
struct LzGeom {               // Q32 map of canvas (i, j) to the source point, Eq. (2) with the scale in (cq, sq)
    long long cq, sq, ox, oy;
    int Wr, Hr;
    __device__ __forceinline__ void map(int i, int j, long long &px, long long &py) const
    {
        const long long dx2 = 2LL * i - Wr + 1, dy2 = 2LL * j - Hr + 1;
        px = cq * dx2 + sq * dy2 + ox;
        py = -sq * dx2 + cq * dy2 + oy;
    }
};

constexpr int kLzRowsPerThread = 4;

// Normalised Lanczos-a weights of taps floor(p) - a + 1 .. floor(p) + a at
// fraction f (the top 24 bits of the Q32 fraction): L(x) = sinc(x) sinc(x/a)
// = a sin(pi x) sin(pi x / a) / (pi x)^2, L(0) = 1.
template <int A>
__device__ __forceinline__ void lanczos_weights(uint32_t frac, float *w)
{
    const float f = (float)(frac >> 8) * (1.0f / 16777216.0f);
    float sum = 0.f;
#pragma unroll
    for (int m = -A + 1; m <= A; ++m) {
        const float x = f - (float)m;
        float L = 1.f;
        if (x != 0.f) {
            const float px = 3.14159265358979f * x;
            L = (float)A * sinpif(x) * sinpif(x * (1.0f / (float)A)) / (px * px);
        }
        w[m + A - 1] = L;
        sum += L;
    }
    const float inv = 1.0f / sum;
#pragma unroll
    for (int k = 0; k < 2 * A; ++k) w[k] *= inv;
}
}  // namespace

template <int A>
__device__ __forceinline__ void warp_lz_tile(int tile, const DevView *__restrict__ views, int n_views, int cwp,
                                             uint8_t *__restrict__ out_u8, uint8_t *__restrict__ out_mask,
                                             float *__restrict__ out_f32)
{
    extern __shared__ float4 smem4[];
    float *Cs = reinterpret_cast<float *>(smem4);      // [kWarpTH][cwp] canvas strip
    float *Bs = Cs + kWarpTH * cwp;                    // [kWarpTH][cwp] blurred strip
    float *gs = Bs + kWarpTH * cwp;                    // Gaussian taps g_0 .. g_K

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
    const LzGeom G{V.cq, V.sq, (long long)(W - 1) * HALF, (long long)(H - 1) * HALF, Wr, V.Hr};

    const long long Xa = V.tq * (2LL * xa - V.Wv + 1) + xoff;
    const long long Xb = V.tq * (2LL * xb - V.Wv + 1) + xoff;
    // B at canvas columns [bl, bh] (the tilt taps, clamped); C over their Gaussian windows
    const int bl = clampi((int)(Xa >> 32) - A + 1, 0, Wr - 1), bh = clampi((int)(Xb >> 32) + A, 0, Wr - 1);
    const int nb = min(bh - bl + 1, cwp);
    const int cl = max(0, bl - K);
    const int nc = min(min(Wr - 1, bh + K) - cl + 1, cwp);    // never above cwp: see warp_lz_strip_width

    for (int k = threadIdx.x; k <= K; k += blockDim.x) gs[k] = V.g[k];

    const int rg4 = (int)(threadIdx.x / 64u) * kLzRowsPerThread;
    // 1. canvas strip
    {
        const long long xlim = (long long)(2 * W - 1) * HALF, ylim = (long long)(2 * H - 1) * HALF;
        const long long dpx = 2LL * V.sq, dpy = 2LL * V.cq;
        const float *__restrict__ src = V.src;
        const int sp = V.src_pitch;
        for (int c = (int)(threadIdx.x & 63u); c < nc; c += 64) {
            long long px, py;
            G.map(cl + c, j0 + rg4, px, py);
            for (int q = 0; q < kLzRowsPerThread; ++q, px += dpx, py += dpy) {
                const int r = rg4 + q;
                if (r >= nrows) break;
                float val = 0.f;
                if (px >= -HALF && px < xlim && py >= -HALF && py < ylim) {
                    float wx[2 * A], wy[2 * A];
                    lanczos_weights<A>((uint32_t)px, wx);
                    lanczos_weights<A>((uint32_t)py, wy);
                    const int x0 = (int)(px >> 32), y0 = (int)(py >> 32);
                    int xs[2 * A];
#pragma unroll
                    for (int m = 0; m < 2 * A; ++m) xs[m] = clampi(x0 - A + 1 + m, 0, W - 1);
#pragma unroll
                    for (int n = 0; n < 2 * A; ++n) {
                        const float *row = src + (size_t)clampi(y0 - A + 1 + n, 0, H - 1) * sp;
                        float acc = 0.f;
#pragma unroll
                        for (int m = 0; m < 2 * A; ++m) acc = fmaf(wx[m], __ldg(row + xs[m]), acc);
                        val = fmaf(wy[n], acc, val);
                    }
                }
                Cs[r * cwp + c] = val;
            }
        }
    }
    __syncthreads();

    // 2. Gaussian along x at the B columns
    for (int b = (int)(threadIdx.x & 63u); b < nb; b += 64) {
        const int i = bl + b;
        for (int q = 0; q < kLzRowsPerThread; ++q) {
            const int r = rg4 + q;
            if (r >= nrows) break;
            const float *Cr = Cs + r * cwp;
            float acc = 0.f;
            if (i - K >= 0 && i + K <= Wr - 1) {
                for (int k = -K; k <= K; ++k) acc = fmaf(gs[abs(k)], Cr[i - k - cl], acc);
            } else {
                for (int k = -K; k <= K; ++k) acc = fmaf(gs[abs(k)], Cr[clampi(i - k, 0, Wr - 1) - cl], acc);
            }
            Bs[r * cwp + b] = acc;
        }
    }
    __syncthreads();

    // 3. Lanczos-a tilt, quantisation and the footprint mask
    {
        const int c = (int)(threadIdx.x & 63u), rg = (int)(threadIdx.x / 64u);
        const int ncols = xb - xa + 1;
        constexpr int kRowStep = kWarpThreads / 64;
        if (c < ncols) {
            const int x = xa + c;
            const long long X = V.tq * (2LL * x - V.Wv + 1) + xoff;
            const int x0 = (int)(X >> 32);
            float w[2 * A];
            lanczos_weights<A>((uint32_t)X, w);
            int bi[2 * A];
#pragma unroll
            for (int m = 0; m < 2 * A; ++m) bi[m] = clampi(x0 - A + 1 + m, 0, Wr - 1) - bl;
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
                const float *Br = Bs + r * cwp;
                float v = 0.f;
#pragma unroll
                for (int m = 0; m < 2 * A; ++m) v = fmaf(w[m], Br[bi[m]], v);
                const int j = j0 + r;
                const bool valid = cols_ok && pxa >= mxlo && pxa <= mxhi && pya >= mylo && pya <= myhi &&
                                   pxb >= mxlo && pxb <= mxhi && pyb >= mylo && pyb <= myhi;
                const size_t o = (size_t)V.out_off + (size_t)j * V.Wv + x;
                if (out_f32) out_f32[o] = v;
                out_u8[o] = (uint8_t)min(255, max(0, __float2int_rn(v)));
                out_mask[o] = (uint8_t)valid;
            }
        }
    }
}

template <int A>
__global__ void __launch_bounds__(kWarpThreads)
warp_lz_kernel(int n_tiles, const DevView *__restrict__ views, int n_views, int cwp, uint8_t *__restrict__ out_u8,
               uint8_t *__restrict__ out_mask, float *__restrict__ out_f32)
{
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        warp_lz_tile<A>(tile, views, n_views, cwp, out_u8, out_mask, out_f32);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side
// Columns of the canvas strip for a tile of tw view columns: the tilt taps of
// the first and last view columns lie t (tw - 1) (+ the Q31 rounding of t)
// apart, plus a - 1 and a on either side, plus K for the Gaussian.
int warp_lz_strip_width(const asift_view_desc &v, int tw, int a)
{
    return (int)std::ceil(v.t * (tw - 1)) + 2 + 2 * a + 2 * v.K;
}

cudaError_t launch_warp_lanczos(int a, const DevView *d_views, int n_views, int n_tiles, int cw_max, uint8_t *u8,
                                uint8_t *mask, float *f32, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    if (a != 3 && a != 4) return cudaErrorInvalidValue;
    const int cwp = cw_max | 1;
    const size_t smem = sizeof(float) * (2 * (size_t)kWarpTH * cwp + ASIFT_MAX_GAUSS);
    const void *fn = a == 4 ? (const void *)warp_lz_kernel<4> : (const void *)warp_lz_kernel<3>;
    const cudaError_t e = ensure_dynamic_smem(fn, smem);
    if (e != cudaSuccess) return e;
    if (a == 4)
        warp_lz_kernel<4><<<n_tiles, kWarpThreads, smem, s>>>(n_tiles, d_views, n_views, cwp, u8, mask, f32);
    else
        warp_lz_kernel<3><<<n_tiles, kWarpThreads, smem, s>>>(n_tiles, d_views, n_views, cwp, u8, mask, f32);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asift
