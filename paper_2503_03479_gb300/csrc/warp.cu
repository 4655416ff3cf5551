// warp.cu -- affine view simulation (Eq. (2)-(4)) on sm_103a.
//
// One CTA produces a kWarpTW x kWarpTH tile of one view.  A view row j only
// depends on canvas row j (the tilt acts along canvas x), so the tile needs a
// canvas strip of kWarpTH rows and columns [bx0 - K, bx1 + K], where
// [bx0, bx1] = [floor(X(x'_first)) - 2, floor(X(x'_last)) + 3] are the columns
// the tilt taps read.  The CTA:
//   1. computes the rotated canvas C on that strip in chunks of kChunk
//      columns; for each chunk the source pixels its 6x6 Lanczos-3 taps can
//      reach (the bounding box of the rotated chunk, at most 72 x 72) are
//      first staged in shared memory, so every tap is a shared-memory load
//      (Eq. (3)-(4); geometry in exact Q32 fixed point);
//   2. blurs the strip along x with the Gaussian taps (B), four outputs per
//      thread so each loaded C value serves four sums;
//   3. resamples B at X = t (x' - (Wv-1)/2) + (Wr-1)/2 with Lanczos-3 and
//      writes fp32 (optional), rint-to-u8 and the footprint mask.
// Strip position i holds the value of canvas column clamp(i, 0, Wr-1), which
// realises the clamped borders of the Gaussian and of the tilt taps without
// per-tap clamps.
// Every launch covers a list of views (one view for the per-view form, all
// views of several images for the batched form); a CTA finds its view by a
// binary search over the views' first tile index.
#include "common.cuh"
#include "kernels.h"

namespace asift {

constexpr int kChunk = 64;              // canvas columns per staged chunk
constexpr int kStage = 80;              // staged source box (rows, columns), >= 64|c| + 16|s| + 6
constexpr int kStagePitch = kStage + 1; // odd pitch against bank conflicts

// sin and cos on [0, pi/3] from their Taylor series (truncation below 5e-8).
__device__ __forceinline__ void sincos_small(float x, float &s, float &c)
{
    const float x2 = x * x;
    s = x * fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 2.75573192e-6f, -1.98412698e-4f), 8.33333333e-3f),
                          -1.66666667e-1f), 1.0f);
    c = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, -2.75573192e-7f, 2.48015873e-5f), -1.38888889e-3f),
                                4.16666667e-2f), -0.5f), 1.0f);
}

// Normalised Lanczos-3 weights (Eq. (4), a = 3) of the taps floor(p) + m,
// m = -2..3, at fractional position f in [0, 1) given as Q32 bits `lo`.
// L(f - m) = 3 sin(pi (f - m)) sin(pi (f - m)/3) / (pi (f - m))^2 and
// sin(pi (f - m)) = (-1)^m sin(pi f): the common factor 3 sin(pi f)/pi^2
// cancels in the normalisation, leaving
//   w_m  ~  (-1)^m sin(pi f/3 - pi m/3) / (f - m)^2,
// whose six sines follow from sin and cos of pi f/3 by angle addition.
// f = 0 (lo == 0) is the identity.
__device__ __forceinline__ void lanczos3_weights(uint32_t lo, float w[6])
{
    if (lo == 0u) {
        w[0] = w[1] = w[3] = w[4] = w[5] = 0.f;
        w[2] = 1.f;
        return;
    }
    const float f = __uint2float_rz(lo) * 2.3283064365386963e-10f;   // < 1
    float s, c;
    sincos_small(f * 1.04719755119659775f, s, c);
    const float hs = 0.5f * s, hc = 0.86602540378443864676f * c;
    const float a = hc - hs, b = -(hs + hc);
    const float d0 = f + 2.f, d1 = f + 1.f, d3 = f - 1.f, d4 = f - 2.f, d5 = f - 3.f;
    const float w0 = __fdividef(a, d0 * d0), w1 = __fdividef(b, d1 * d1), w2 = __fdividef(s, f * f);
    const float w3 = __fdividef(a, d3 * d3), w4 = __fdividef(b, d4 * d4), w5 = __fdividef(s, d5 * d5);
    const float inv = __frcp_rn(((w0 + w1) + (w2 + w3)) + (w4 + w5));
    w[0] = w0 * inv; w[1] = w1 * inv; w[2] = w2 * inv;
    w[3] = w3 * inv; w[4] = w4 * inv; w[5] = w5 * inv;
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

// Every image of a list: blockIdx.y selects the image, x strides its pixels.
__global__ void convert_images_kernel(const ImageConv *__restrict__ list)
{
    const ImageConv c = list[blockIdx.y];
    const long long n = (long long)c.W * c.H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / c.W), x = (int)(i - (long long)y * c.W);
        c.dst[i] = (float)c.src[(size_t)y * c.pitch + x];
    }
}

struct CanvasGeom {           // Q32 map of canvas (i, j) to the source point
    long long cq, sq, ox, oy;  // p = (cq*dx2 + sq*dy2 + ox, -sq*dx2 + cq*dy2 + oy)
    int Wr, Hr;
    __device__ __forceinline__ void map(int i, int j, long long &px, long long &py) const
    {
        const long long dx2 = 2LL * i - Wr + 1, dy2 = 2LL * j - Hr + 1;
        px = cq * dx2 + sq * dy2 + ox;
        py = -sq * dx2 + cq * dy2 + oy;
    }
};

__device__ __forceinline__ void warp_view_tile(int tile, const DevView *__restrict__ views, int n_views, int cw_max, int bw_max,
                 uint8_t *__restrict__ out_u8, uint8_t *__restrict__ out_mask, float *__restrict__ out_f32)
{
    extern __shared__ float smem[];
    float *Cs = smem;                              // [kWarpTH][cw_max]
    float *Bs = Cs + kWarpTH * cw_max;             // [kWarpTH][bw_max]
    float *Ss = Bs + kWarpTH * bw_max;             // [kStage][kStagePitch] staged source
    __shared__ float gs[ASIFT_MAX_GAUSS];

    const int vi = find_owner(views, n_views, tile, [](const DevView &v) { return v.tile_start; });
    const DevView &V = views[vi];
    const int lt = tile - V.tile_start;
    const int ty = lt / V.ntx, tx = lt - ty * V.ntx;
    const int xa = tx * kWarpTW, xb = min(xa + kWarpTW, V.Wv) - 1;
    const int j0 = ty * kWarpTH, j1 = min(j0 + kWarpTH, V.Hv) - 1;
    const int nrows = j1 - j0 + 1;
    const int Wr = V.Wr, K = V.K, W = V.W, H = V.H;
    const long long HALF = 2147483648LL;
    const long long xoff = (long long)(Wr - 1) * HALF;
    const CanvasGeom G{V.cq, V.sq, (long long)(W - 1) * HALF, (long long)(H - 1) * HALF, Wr, V.Hr};

    const long long Xa = V.tq * (2LL * xa - V.Wv + 1) + xoff;
    const long long Xb = V.tq * (2LL * xb - V.Wv + 1) + xoff;
    const int bx0 = (int)(Xa >> 32) - 2, bx1 = (int)(Xb >> 32) + 3;   // unclamped strip of B
    const int bw = bx1 - bx0 + 1;
    const int cx0 = bx0 - K;                // strip of C: [cx0, cx0 + cw), covering the Gaussian
    const int cw = ((bw + 3) & ~3) + 2 * K; // taps of B computed four at a time

    for (int k = threadIdx.x; k <= K; k += blockDim.x) gs[k] = V.g[k];

    // 1. rotated canvas strip, chunk by chunk through shared memory
    const float *__restrict__ src = V.src;
    const int sp = V.src_pitch;
    const long long xlim = (long long)(2 * W - 1) * HALF, ylim = (long long)(2 * H - 1) * HALF;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < cw; c0 += kChunk) {
        const int cn = min(kChunk, cw - c0);
        // source box of this chunk: the taps of the four corners of the
        // (clamped) canvas region, clamped to the image
        const int i_lo = clampi(cx0 + c0, 0, Wr - 1), i_hi = clampi(cx0 + c0 + cn - 1, 0, Wr - 1);
        int sx0 = 1 << 30, sx1 = -(1 << 30), sy0 = 1 << 30, sy1 = -(1 << 30);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            long long px, py;
            G.map(q & 1 ? i_hi : i_lo, q & 2 ? j1 : j0, px, py);
            sx0 = min(sx0, (int)(px >> 32));
            sx1 = max(sx1, (int)(px >> 32));
            sy0 = min(sy0, (int)(py >> 32));
            sy1 = max(sy1, (int)(py >> 32));
        }
        sx0 = clampi(sx0 - 2, 0, W - 1);
        sx1 = clampi(sx1 + 3, 0, W - 1);
        sy0 = clampi(sy0 - 2, 0, H - 1);
        sy1 = clampi(sy1 + 3, 0, H - 1);
        // a chunk spans at most 63 columns and 15 rows of the canvas, so the
        // box spans at most sqrt(63^2 + 15^2) + 1 + 5 < 73 <= kStage source pixels
        const int bwid = sx1 - sx0 + 1, bhgt = sy1 - sy0 + 1;
        __syncthreads();   // previous chunk's reads of Ss are done
        for (int r = warp; r < bhgt; r += kWarpThreads / 32) {
            const float *srow = src + (size_t)(sy0 + r) * sp + sx0;
            for (int c = lane; c < bwid; c += 32) Ss[r * kStagePitch + c] = __ldg(srow + c);
        }
        __syncthreads();
        // canvas pixels of the chunk; a warp covers 8 columns x 4 rows so its
        // lanes' taps fall in a compact source region
        const int nblk_c = (cn + 7) >> 3, nblk_r = (nrows + 3) >> 2;
        for (int blk = warp; blk < nblk_c * nblk_r; blk += kWarpThreads / 32) {
            const int c = ((blk % nblk_c) << 3) + (lane & 7u);
            const int r = ((blk / nblk_c) << 2) + (lane >> 3);
            if (c >= cn || r >= nrows) continue;
            const int i = clampi(cx0 + c0 + c, 0, Wr - 1), j = j0 + r;
            long long px, py;
            G.map(i, j, px, py);
            float acc = 0.f;
            if (px >= -HALF && px < xlim && py >= -HALF && py < ylim) {
                float wx[6], wy[6];
                lanczos3_weights((uint32_t)px, wx);
                lanczos3_weights((uint32_t)py, wy);
                const int x0 = (int)(px >> 32), y0 = (int)(py >> 32);
                if (x0 >= 2 && x0 + 3 < W && y0 >= 2 && y0 + 3 < H) {
                    // interior: no clamped taps, one base address and immediate offsets
                    const float *b = Ss + (y0 - 2 - sy0) * kStagePitch + (x0 - 2 - sx0);
                    float rs[6];
#pragma unroll
                    for (int n = 0; n < 6; ++n) {
                        const float *row = b + n * kStagePitch;
                        rs[n] = fmaf(wx[0], row[0], fmaf(wx[1], row[1], fmaf(wx[2], row[2],
                                fmaf(wx[3], row[3], fmaf(wx[4], row[4], wx[5] * row[5])))));
                    }
                    acc = fmaf(wy[0], rs[0], fmaf(wy[1], rs[1], fmaf(wy[2], rs[2],
                          fmaf(wy[3], rs[3], fmaf(wy[4], rs[4], wy[5] * rs[5])))));
                } else {
                    int xs[6];
#pragma unroll
                    for (int m = 0; m < 6; ++m) xs[m] = clampi(x0 + m - 2, 0, W - 1) - sx0;
#pragma unroll
                    for (int n = 0; n < 6; ++n) {
                        const float *row = Ss + (clampi(y0 + n - 2, 0, H - 1) - sy0) * kStagePitch;
                        float a = 0.f;
#pragma unroll
                        for (int m = 0; m < 6; ++m) a = fmaf(wx[m], row[xs[m]], a);
                        acc = fmaf(wy[n], a, acc);
                    }
                }
            }
            Cs[r * cw_max + c0 + c] = acc;
        }
    }
    __syncthreads();

    // 2. Gaussian along canvas x: B(i) = sum_k g_|k| C(clamp(i) - k), four
    //    consecutive outputs per thread.  Strip index of canvas column i is
    //    i - cx0; clamp(i) - k stays inside [cx0, cx0 + cw).
    const int nq4 = (bw + 3) >> 2;
    for (int e = threadIdx.x; e < nrows * nq4; e += blockDim.x) {
        const int r = e / nq4, q4 = e - r * nq4;
        const float *Crow = Cs + r * cw_max - cx0;
        float *Brow = Bs + r * bw_max - bx0;
        const int ib = bx0 + 4 * q4;
        const int ic0 = clampi(ib, 0, Wr - 1), ic1 = clampi(ib + 1, 0, Wr - 1);
        const int ic2 = clampi(ib + 2, 0, Wr - 1), ic3 = clampi(ib + 3, 0, Wr - 1);
        if (ic3 - ic0 == 3) {       // interior: a sliding window shared by the four outputs
            float a0 = gs[0] * Crow[ic0], a1 = gs[0] * Crow[ic0 + 1];
            float a2 = gs[0] * Crow[ic0 + 2], a3 = gs[0] * Crow[ic0 + 3];
            for (int k = 1; k <= K; ++k) {
                const float g = gs[k];
                const float l0 = Crow[ic0 - k], l1 = Crow[ic0 + 1 - k], l2 = Crow[ic0 + 2 - k], l3 = Crow[ic0 + 3 - k];
                const float h0 = Crow[ic0 + k], h1 = Crow[ic0 + 1 + k], h2 = Crow[ic0 + 2 + k], h3 = Crow[ic0 + 3 + k];
                a0 = fmaf(g, l0 + h0, a0);
                a1 = fmaf(g, l1 + h1, a1);
                a2 = fmaf(g, l2 + h2, a2);
                a3 = fmaf(g, l3 + h3, a3);
            }
            Brow[ib] = a0;
            if (ib + 1 <= bx1) Brow[ib + 1] = a1;
            if (ib + 2 <= bx1) Brow[ib + 2] = a2;
            if (ib + 3 <= bx1) Brow[ib + 3] = a3;
        } else {                    // the canvas border: each output on its own
            const int icq[4] = {ic0, ic1, ic2, ic3};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (ib + q > bx1) break;
                const int ic = icq[q];
                float a = gs[0] * Crow[ic];
                for (int k = 1; k <= K; ++k) a = fmaf(gs[k], Crow[ic - k] + Crow[ic + k], a);
                Brow[ib + q] = a;
            }
        }
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
        for (int m = 0; m < 6; ++m) v = fmaf(w[m], Brow[x0 + m - 2], v);
        int valid = 1;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = x0 + q;
            if (i < 0 || i >= Wr) { valid = 0; continue; }
            long long px, py;
            G.map(i, j, px, py);
            valid &= (px >= mxlo && px <= mxhi && py >= mylo && py <= myhi);
        }
        const size_t o = (size_t)V.out_off + (size_t)j * V.Wv + x;
        if (out_f32) out_f32[o] = v;
        const int q8 = __float2int_rn(v);
        out_u8[o] = (uint8_t)min(255, max(0, q8));
        out_mask[o] = (uint8_t)valid;
    }
}

// Grid-stride over the tiles: one CTA per tile, or a persistent grid.
__global__ void __launch_bounds__(kWarpThreads, 3)
warp_view_kernel(int n_tiles, const DevView *__restrict__ views, int n_views, int cw_max, int bw_max,
                 uint8_t *__restrict__ out_u8, uint8_t *__restrict__ out_mask, float *__restrict__ out_f32)
{
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        warp_view_tile(tile, views, n_views, cw_max, bw_max, out_u8, out_mask, out_f32);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side
void warp_strip_widths(const asift_view_desc &v, int *cw, int *bw)
{
    // B strip: floor(X) - 2 .. floor(X) + 3 over kWarpTW view columns spaced
    // t apart (+1 for the rounding of tq); C strip adds K on both sides.
    const int span = (int)std::ceil(v.t * (kWarpTW - 1)) + 2;
    *bw = span + 6;
    *cw = ((*bw + 3) & ~3) + 2 * v.K;
}

size_t warp_smem_bytes(int cw_max, int bw_max)
{
    return sizeof(float) * ((size_t)kWarpTH * (cw_max + bw_max) + (size_t)kStage * kStagePitch);
}

cudaError_t launch_u8_to_f32(const uint8_t *src, int pitch, int W, int H, float *dst, cudaStream_t s)
{
    const long long n = (long long)W * H;
    int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
    u8_to_f32_kernel<<<blocks, 256, 0, s>>>(src, pitch, W, H, dst);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_convert_images(const ImageConv *d_list, int n, long long max_px, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int bx = (int)std::max<long long>(1, std::min<long long>((max_px + 255) / 256, 152LL * 4));
    convert_images_kernel<<<dim3(bx, n), 256, 0, s>>>(d_list);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_warp(const DevView *d_views, int n_views, int n_tiles, int cw_max, int bw_max,
                        uint8_t *u8, uint8_t *mask, float *f32, cudaStream_t s, int grid)
{
    if (n_tiles <= 0) return cudaSuccess;
    const size_t smem = warp_smem_bytes(cw_max, bw_max);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(warp_view_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int g = (grid > 0 && grid < n_tiles) ? grid : n_tiles;
    warp_view_kernel<<<g, kWarpThreads, smem, s>>>(n_tiles, d_views, n_views, cw_max, bw_max, u8, mask, f32);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asift
