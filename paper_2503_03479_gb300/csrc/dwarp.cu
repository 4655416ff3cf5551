// dwarp.cu -- the differentiable view warp and its backward on sm_103a (the
// photometric refinement path of the best simulated view).
//
// Forward: the chain of Eq. (2)-(4) with continuous parameters
// theta = (t, phi, tx, ty): canvas C(i, j) = normalised Lanczos-3 sample of u
// at p = R(phi)^T ((i, j) - c_r) + c_s + (tx, ty) with every tap clamped to the
// image; B = Gaussian (sigma = 0.8 sqrt(t^2 - 1), fixed half width K) along
// canvas x; v(x', j) = Lanczos-3 sample of B's row j at
// X = t (x' - (Wv-1)/2) + (Wr-1)/2.  Canvas and view sizes are fixed.
//
// Backward (one CTA per view tile, no state kept from the forward): the canvas
// strip C, its derivatives dC/dp (one weight evaluation) and its blur B are
// recomputed in shared memory; the tile's part of B-bar (the tilt transposed)
// is gathered per strip position, folded onto canvas columns, and C-bar (the
// Gaussian transposed) gathered from it; C-bar drives the parameter
// derivatives through the stored dC/dp and, when the image gradient is asked
// for, scatters into u-bar (the rotation transposed) through shared-memory
// patches flushed with global atomics.  Tiles only add partial adjoints, so
// the sum over tiles is the exact transpose (up to fp32 summation order).
#include "common.cuh"
#include "kernels.h"

namespace asift {

// Tiles of kDTH view rows x tw view columns, tw = 64 in both directions: the
// canvas strip of a tile, t (tw - 1) + 8 + 2K columns, then recomputes a
// smaller share of halo per view pixel.  (The backward's five strips per row
// then hold two CTAs per SM instead of three with tw = 32; measured on 256
// views of 512^2 it still gains 6% with the image gradient and is level
// without.)
constexpr int kDTWFwd = 64, kDTWBwd = 64, kDTH = 8, kDThreads = 256;
constexpr int kBcPad = ASIFT_MAX_GAUSS;   // zero columns either side of a folded B-bar row (> K)

// sinc(x) and sinc(x/3) with their x-derivatives near x = 0 (|x| < 1e-2),
// where the closed forms cancel: the series to (pi x)^4.
__device__ __forceinline__ void sinc_series(float x, float &a, float &da, float &b, float &db)
{
    const float y = 9.8696044010893586f * x * x;   // (pi x)^2
    a = 1.f - y * (1.f / 6.f) * (1.f - y * (1.f / 20.f));
    da = -3.2898681336964529f * x * (1.f - y * (1.f / 10.f));   // -(pi^2 x / 3)(1 - (pi x)^2/10)
    const float y3 = y * (1.f / 9.f);                            // (pi x / 3)^2
    b = 1.f - y3 * (1.f / 6.f) * (1.f - y3 * (1.f / 20.f));
    db = -0.36554090374405032f * x * (1.f - y3 * (1.f / 10.f));  // -(pi^2 x / 27)(1 - (pi x/3)^2/10)
}

// Lanczos-3 kernel L(x) = sinc(x) sinc(x/3) (Eq. (4), a = 3) at the six taps
// x = f - m', m' = -2..3 (index m = m' + 2), and L'(x) when D is true.  One
// sincospif pair serves all six: sin(pi x) = (-1)^m' sin(pi f), cos likewise,
// and sin, cos of pi x/3 follow from those of pi f/3 by angle addition with
// the constants cos, sin of pi m'/3.  With r = 1/x:
//   sinc(x)   = sin(pi x) r / pi,      d/dx = (cos(pi x) - sinc(x)) r,
//   sinc(x/3) = 3 sin(pi x/3) r / pi,  d/dx = (cos(pi x/3) - sinc(x/3)) r.
// Outside |x| < 3 (only x = -3, at f = 0) the kernel and its derivative are 0.
template <bool D>
__device__ __forceinline__ void lanczos3_taps(float f, float L[6], float dL[6])
{
    constexpr float kR3 = 0.86602540378443864676f;
    constexpr float kCos[6] = {-0.5f, 0.5f, 1.f, 0.5f, -0.5f, -1.f};
    constexpr float kSin[6] = {-kR3, -kR3, 0.f, kR3, kR3, 0.f};
    float S1, C1, S3, C3;
    sincospif(f, &S1, &C1);
    sincospif(f * (1.f / 3.f), &S3, &C3);
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const float x = f - (float)(m - 2);
        const float sx = (m & 1) ? -S1 : S1, cx = (m & 1) ? -C1 : C1;
        const float s3 = fmaf(S3, kCos[m], -C3 * kSin[m]);
        const float c3 = fmaf(C3, kCos[m], S3 * kSin[m]);
        const bool small = fabsf(x) < 1e-2f;
        const float r = __frcp_rn(small ? 1.f : x);
        float a = sx * r * 0.31830988618379067f, b = s3 * r * 0.95492965855137202f;
        float da = 0.f, db = 0.f;
        if (D) {
            da = (cx - a) * r;
            db = (c3 - b) * r;
        }
        if (small) {
            float sa, sda, sb, sdb;
            sinc_series(x, sa, sda, sb, sdb);
            a = sa; b = sb; da = sda; db = sdb;
        }
        const bool in = fabsf(x) < 3.f;
        L[m] = in ? a * b : 0.f;
        if (D) dL[m] = in ? fmaf(da, b, a * db) : 0.f;
    }
}

// Normalised Lanczos-3 weights w_m(f) (m = -2..3) and dw_m/df, the quotient
// rule on w_m = L_m / sum_n L_n (the forward and the backward share them).
__device__ __forceinline__ void lanczos3_wd(float f, float w[6], float dw[6])
{
    float L[6], dL[6];
    lanczos3_taps<true>(f, L, dL);
    const float S = ((L[0] + L[1]) + (L[2] + L[3])) + (L[4] + L[5]);
    const float dS = ((dL[0] + dL[1]) + (dL[2] + dL[3])) + (dL[4] + dL[5]);
    const float inv = 1.f / S;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        w[m] = L[m] * inv;
        dw[m] = (dL[m] - w[m] * dS) * inv;
    }
}

// The weights alone.
__device__ __forceinline__ void lanczos3_w(float f, float w[6])
{
    float L[6], dL[6];
    lanczos3_taps<false>(f, L, dL);
    const float inv = 1.f / (((L[0] + L[1]) + (L[2] + L[3])) + (L[4] + L[5]));
#pragma unroll
    for (int m = 0; m < 6; ++m) w[m] = L[m] * inv;
}

struct DGeom {
    float c, s, cx, cy, tx, ty, crx, cry;
    __device__ __forceinline__ void map(int i, int j, float &px, float &py) const
    {
        const float dx = (float)i - crx, dy = (float)j - cry;
        px = fmaf(c, dx, fmaf(s, dy, cx + tx));
        py = fmaf(-s, dx, fmaf(c, dy, cy + ty));
    }
};

// Canvas value at p (taps clamped to the image), optionally with dC/dpx and
// dC/dpy.
__device__ __forceinline__ float canvas_at(const float *__restrict__ u, int W, int H, float px, float py,
                                           float *dcdx, float *dcdy)
{
    const float fx0 = floorf(px), fy0 = floorf(py);
    const int x0 = (int)fx0, y0 = (int)fy0;
    float wx[6], dwx[6], wy[6], dwy[6];
    if (dcdx) {
        lanczos3_wd(px - fx0, wx, dwx);
        lanczos3_wd(py - fy0, wy, dwy);
    } else {
        lanczos3_w(px - fx0, wx);
        lanczos3_w(py - fy0, wy);
    }
    int xs[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) xs[m] = clampi(x0 + m - 2, 0, W - 1);
    float acc = 0.f, ax = 0.f, ay = 0.f;
#pragma unroll
    for (int n = 0; n < 6; ++n) {
        const float *row = u + (size_t)clampi(y0 + n - 2, 0, H - 1) * W;
        float r = 0.f, dr = 0.f;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const float val = __ldg(row + xs[m]);
            r = fmaf(wx[m], val, r);
            if (dcdx) dr = fmaf(dwx[m], val, dr);
        }
        acc = fmaf(wy[n], r, acc);
        if (dcdx) {
            ax = fmaf(wy[n], dr, ax);
            ay = fmaf(dwy[n], r, ay);
        }
    }
    if (dcdx) {
        *dcdx = ax;
        *dcdy = ay;
    }
    return acc;
}

// u-bar += cb w_x w_y over the 6 x 6 taps of p (the rotation's sample
// transposed; clamped taps add at the edge pixels they read).  Where the six
// columns lie inside the image and the rows' 16-byte groups inside the row
// (W a multiple of 4), each tap row is two or three float4 reductions over
// the aligned groups that hold it (zeros on either side), else six scalar ones.
__device__ __forceinline__ void scatter_ubar(float *__restrict__ ubar, int W, int H, float px, float py, float cb)
{
    const float fx0 = floorf(px), fy0 = floorf(py);
    const int x0 = (int)fx0, y0 = (int)fy0;
    float wx[6], wy[6];
    lanczos3_w(px - fx0, wx);
    lanczos3_w(py - fy0, wy);
    const int xa = x0 - 2, a = xa & ~3, o = xa - a;   // first tap, its group, offset in the group
    const int ng = o == 3 ? 3 : 2;
    if ((W & 3) == 0 && xa >= 0 && a + 4 * ng <= W) {
        // the weights shifted to their lanes in the groups: lane j holds tap j - o
        float sw[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            float v = 0.f;
#pragma unroll
            for (int m = 0; m < 6; ++m) v = (j - m == o) ? wx[m] : v;
            sw[j] = v;
        }
#pragma unroll
        for (int n = 0; n < 6; ++n) {
            const float cn = cb * wy[n];
            float4 *row = reinterpret_cast<float4 *>(ubar + (size_t)clampi(y0 + n - 2, 0, H - 1) * W + a);
            atomicAdd(row, make_float4(cn * sw[0], cn * sw[1], cn * sw[2], cn * sw[3]));
            atomicAdd(row + 1, make_float4(cn * sw[4], cn * sw[5], cn * sw[6], cn * sw[7]));
            if (ng == 3) atomicAdd(row + 2, make_float4(cn * sw[8], 0.f, 0.f, 0.f));
        }
        return;
    }
    int xs[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) xs[m] = clampi(x0 + m - 2, 0, W - 1);
#pragma unroll
    for (int n = 0; n < 6; ++n) {
        float *row = ubar + (size_t)clampi(y0 + n - 2, 0, H - 1) * W;
        const float cn = cb * wy[n];
#pragma unroll
        for (int m = 0; m < 6; ++m) atomicAdd(row + xs[m], cn * wx[m]);
    }
}

// A u-bar patch: a block of 32 canvas columns x 8 rows spans at most
// sqrt(31^2 + 7^2) + 1 < 33 source pixels along either axis, + 5 for the taps
// and 2 of margin.  The odd row pitch spreads a warp's taps along a steep
// line of source rows over the banks.
constexpr int kPatch = 40, kPatchPitch = 41;

// u-bar += cb w_x w_y over the taps of p, into the patch whose pixel (0, 0)
// is source (bx0, by0), in fixed point: each product is rounded to a multiple
// of 1/scale and added with a shared-memory integer atomic (exact and in
// any order, where float adds would need compare-and-swap loops); a tap
// outside the patch, which its box construction rules out, goes to u-bar
// directly.
__device__ __forceinline__ void scatter_patch(int *P, int bx0, int by0, int PW, int PH, float scale,
                                              float *__restrict__ ubar, int W, int H, float px, float py, float cb)
{
    const float fx0 = floorf(px), fy0 = floorf(py);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int xl = clampi(x0 - 2, 0, W - 1) - bx0, xh = clampi(x0 + 3, 0, W - 1) - bx0;
    const int yl = clampi(y0 - 2, 0, H - 1) - by0, yh = clampi(y0 + 3, 0, H - 1) - by0;
    if (xl < 0 || xh >= PW || yl < 0 || yh >= PH) {
        scatter_ubar(ubar, W, H, px, py, cb);
        return;
    }
    float wx[6], wy[6];
    lanczos3_w(px - fx0, wx);
    lanczos3_w(py - fy0, wy);
    int xs[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) xs[m] = clampi(x0 + m - 2, 0, W - 1) - bx0;
    const float cs = cb * scale;
#pragma unroll
    for (int n = 0; n < 6; ++n) {
        int *row = P + (clampi(y0 + n - 2, 0, H - 1) - by0) * kPatchPitch;
        const float cn = cs * wy[n];
#pragma unroll
        for (int m = 0; m < 6; ++m) atomicAdd(row + xs[m], __float2int_rn(cn * wx[m]));
    }
}

// The largest value of v over the block, in every thread (red: 8 floats,
// free on entry).
__device__ __forceinline__ float block_max_all(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    return m;
}

// One block of 64 threads per view: cos, sin of phi and sigma(t) in fp64,
// the Gaussian taps g_k = exp(-k^2 / (2 sigma^2)) / E over k = -K..K and
// dg_k/dsigma = g_k (k^2 - M2) / sigma^3, M2 = sum_k k^2 g_k (the derivative
// of the normalised taps), so that no tile evaluates them.
__global__ void __launch_bounds__(64)
dwarp_prep_kernel(const DiffView *__restrict__ views, DiffPrep *__restrict__ prep)
{
    __shared__ float red_e[2], red_m[2];
    const DiffView &V = views[blockIdx.x];
    DiffPrep &P = prep[blockIdx.x];
    const double t = V.param[0];
    const float sigma = t > 1.0 ? (float)(0.8 * sqrt(t * t - 1.0)) : 0.f;
    const int K = V.K, k = (int)threadIdx.x;
    float v = 0.f;
    if (sigma > 0.f && k <= K) v = expf(-(float)(k * k) / (2.f * sigma * sigma));
    float e = (k == 0) ? v : 2.f * v, m2 = 2.f * v * (float)(k * k);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        m2 += __shfl_xor_sync(0xffffffffu, m2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_e[threadIdx.x >> 5] = e;
        red_m[threadIdx.x >> 5] = m2;
    }
    __syncthreads();
    const float E = red_e[0] + red_e[1], M2 = (red_m[0] + red_m[1]) / E;
    if (k < ASIFT_MAX_GAUSS) {
        if (sigma > 0.f) {
            P.g[k] = k <= K ? v / E : 0.f;
            P.dg[k] = k <= K ? (v / E) * ((float)(k * k) - M2) / (sigma * sigma * sigma) : 0.f;
        } else {
            P.g[k] = (k == 0) ? 1.f : 0.f;
            P.dg[k] = 0.f;
        }
    }
    if (threadIdx.x == 0) {
        const double r = V.param[1] * (3.14159265358979323846 / 180.0);
        P.c = (float)cos(r);
        P.s = (float)sin(r);
        P.sigma = sigma;
        P.pad = 0.f;
        P.dsig_dt = t > 1.0 ? 0.8 * t / sqrt(t * t - 1.0) : 0.0;
    }
}

// The view's Gaussian taps into shared memory.
__device__ __forceinline__ void load_taps(const DiffPrep &P, int K, float *g, float *dg)
{
    for (int k = threadIdx.x; k <= K; k += blockDim.x) {
        g[k] = P.g[k];
        dg[k] = P.dg[k];
    }
}

// A view tile's strips.  B is needed at strip positions bx0..bx1 (the tilt
// taps, unclamped: position i holds B(clamp(i))); C is needed at the actual
// canvas columns clo..chi that the clamped Gaussian taps of those B values
// reach.  When t has grown past the t the sizes were fixed for, a tile's
// positions can all lie beyond the canvas; indexing C by clamped columns keeps
// every shared-memory access inside the strip.
struct DTile {
    int v, xa, xb, j0, j1, bx0, bx1, clo, chi, cw, bw;
    float t, crv;
};

__device__ __forceinline__ DTile dtile(const DiffView *views, int n_views, int tile)
{
    DTile T;
    T.v = find_owner(views, n_views, tile, [](const DiffView &d) { return d.tile_start; });
    const DiffView &V = views[T.v];
    const int lt = tile - V.tile_start;
    const int ty = lt / V.ntx, tx = lt - ty * V.ntx;
    T.xa = tx * V.tw;
    T.xb = min(T.xa + V.tw, V.Wv) - 1;
    T.j0 = ty * kDTH;
    T.j1 = min(T.j0 + kDTH, V.Hv) - 1;
    T.t = (float)V.param[0];
    T.crv = (V.Wv - 1) * 0.5f;
    const float cr = (V.Wr - 1) * 0.5f;
    T.bx0 = (int)floorf(T.t * ((float)T.xa - T.crv) + cr) - 2;
    T.bx1 = (int)floorf(T.t * ((float)T.xb - T.crv) + cr) + 3;
    T.bw = T.bx1 - T.bx0 + 1;
    T.clo = max(0, clampi(T.bx0, 0, V.Wr - 1) - V.K);
    T.chi = min(V.Wr - 1, clampi(T.bx1, 0, V.Wr - 1) + V.K);
    T.cw = T.chi - T.clo + 1;
    return T;
}

__device__ __forceinline__ DGeom dgeom(const DiffView &V, const DiffPrep &P)
{
    DGeom G;
    G.c = P.c;
    G.s = P.s;
    G.cx = (V.W - 1) * 0.5f;
    G.cy = (V.H - 1) * 0.5f;
    G.tx = (float)V.param[2];
    G.ty = (float)V.param[3];
    G.crx = (V.Wr - 1) * 0.5f;
    G.cry = (V.Hr - 1) * 0.5f;
    return G;
}

// The tilt taps of the tile's view columns (one thread per column): X0 =
// floor(X) and the Lanczos-3 weights at X - X0 (with their derivatives when
// dw is given), shared by the tile's rows.
__device__ __forceinline__ void tilt_columns(const DTile &T, float cr, int *X0s, float (*w)[6], float (*dw)[6])
{
    const int ncols = T.xb - T.xa + 1;
    const int c = (int)threadIdx.x;
    if (c < ncols) {
        const float X = T.t * ((float)(T.xa + c) - T.crv) + cr;
        const float fX = floorf(X);
        X0s[c] = (int)fX;
        if (dw) lanczos3_wd(X - fX, w[c], dw[c]);
        else lanczos3_w(X - fX, w[c]);
    }
}

// Recomputes the canvas strip C (actual columns clo..chi) and its blur B
// (strip positions bx0.., value of column clamp(i)) of a tile in shared memory.
__device__ void strips(const DiffView &V, const DTile &T, const DGeom &G, const float *g, float *Cs, float *Bs,
                       int cw_max, int bw_max, float *Cx = nullptr, float *Cy = nullptr)
{
    const int nrows = T.j1 - T.j0 + 1;
    for (int e = threadIdx.x; e < nrows * T.cw; e += blockDim.x) {
        const int r = e / T.cw, c = e - r * T.cw;
        float px, py;
        G.map(T.clo + c, T.j0 + r, px, py);
        if (Cx) {   // with dC/dpx, dC/dpy for the backward (one weight evaluation)
            float dx, dy;
            Cs[r * cw_max + c] = canvas_at(V.u, V.W, V.H, px, py, &dx, &dy);
            Cx[r * cw_max + c] = dx;
            Cy[r * cw_max + c] = dy;
        } else {
            Cs[r * cw_max + c] = canvas_at(V.u, V.W, V.H, px, py, nullptr, nullptr);
        }
    }
    __syncthreads();
    const int last = V.Wr - 1;
    for (int e = threadIdx.x; e < nrows * T.bw; e += blockDim.x) {
        const int r = e / T.bw, c = e - r * T.bw;
        const int ic = clampi(T.bx0 + c, 0, last);
        const float *Crow = Cs + r * cw_max - T.clo;
        float acc = g[0] * Crow[ic];
        for (int k = 1; k <= V.K; ++k) acc = fmaf(g[k], Crow[max(ic - k, 0)] + Crow[min(ic + k, last)], acc);
        Bs[r * bw_max + c] = acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kDThreads)
dwarp_fwd_kernel(const DiffView *__restrict__ views, const DiffPrep *__restrict__ prep, int n_views, int cw_max,
                 int bw_max, int32_t *status)
{
    extern __shared__ float sm[];
    float *Cs = sm, *Bs = sm + kDTH * cw_max;
    __shared__ float g[ASIFT_MAX_GAUSS], dg[ASIFT_MAX_GAUSS];
    const DTile T = dtile(views, n_views, blockIdx.x);
    const DiffView &V = views[T.v];
    if (T.cw > cw_max || T.bw > bw_max || V.K >= ASIFT_MAX_GAUSS) {   // t beyond the t_max the strips were sized for
        if (threadIdx.x == 0) set_status(status, ASIFT_ERR_CAPACITY);
        return;
    }
    const DiffPrep &Pp = prep[T.v];
    const DGeom G = dgeom(V, Pp);
    __shared__ int tX0[kDTWFwd];
    __shared__ float tw[kDTWFwd][6];
    const float cr = (V.Wr - 1) * 0.5f;
    load_taps(Pp, V.K, g, dg);                  // both visible after the
    tilt_columns(T, cr, tX0, tw, nullptr);      // strip's first barrier
    strips(V, T, G, g, Cs, Bs, cw_max, bw_max);
    const int nrows = T.j1 - T.j0 + 1, ncols = T.xb - T.xa + 1;
    for (int e = threadIdx.x; e < nrows * ncols; e += blockDim.x) {
        const int r = e / ncols, c = e - r * ncols;
        const int X0 = tX0[c];
        const float *Brow = Bs + r * bw_max - T.bx0;
        float v = 0.f;
#pragma unroll
        for (int m = 0; m < 6; ++m) v = fmaf(tw[c][m], Brow[X0 + m - 2], v);
        V.out[(size_t)(T.j0 + r) * V.Wv + T.xa + c] = v;
    }
}

__device__ __forceinline__ float block_sum(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;   // valid in thread 0
}

__global__ void __launch_bounds__(kDThreads)
dwarp_bwd_kernel(const DiffView *__restrict__ views, const DiffPrep *__restrict__ prep, int n_views, int cw_max,
                 int bw_max, int32_t *status)
{
    extern __shared__ float sm[];
    float *Cs = sm, *Cx = Cs + kDTH * cw_max, *Cy = Cx + kDTH * cw_max, *Cb = Cy + kDTH * cw_max;
    // B-bar folded onto canvas columns clo .. chi, with kBcPad zero columns either side
    const int bcp = cw_max + 2 * kBcPad;
    float *Bc = Cb + kDTH * cw_max;
    float *Bs = Bc + kDTH * bcp, *Bb = Bs + kDTH * bw_max;
    __shared__ float g[ASIFT_MAX_GAUSS], dg[ASIFT_MAX_GAUSS], red[kDThreads / 32];
    const DTile T = dtile(views, n_views, blockIdx.x);
    const DiffView &V = views[T.v];
    if (T.cw > cw_max || T.bw > bw_max || V.K >= ASIFT_MAX_GAUSS) {
        if (threadIdx.x == 0) set_status(status, ASIFT_ERR_CAPACITY);
        return;
    }
    const DiffPrep &Pp = prep[T.v];
    const DGeom G = dgeom(V, Pp);
    const int K = V.K, last = V.Wr - 1;
    __shared__ int tX0[kDTWBwd];
    __shared__ float tw[kDTWBwd][6], tdw[kDTWBwd][6], vbs[kDTH][kDTWBwd];
    const float cr = (V.Wr - 1) * 0.5f;
    load_taps(Pp, K, g, dg);                    // all visible after the
    tilt_columns(T, cr, tX0, tw, tdw);          // strip's first barrier
    {
        const int ncols = T.xb - T.xa + 1, nrows = T.j1 - T.j0 + 1;
        for (int e = threadIdx.x; e < nrows * ncols; e += blockDim.x) {
            const int r = e / ncols, c = e - r * ncols;
            vbs[r][c] = V.vbar[(size_t)(T.j0 + r) * V.Wv + T.xa + c];
        }
    }
    strips(V, T, G, g, Cs, Bs, cw_max, bw_max, Cx, Cy);
    const int nrows = T.j1 - T.j0 + 1, ncols = T.xb - T.xa + 1;
    // tilt transposed as a gather: strip position P = bx0 + p takes w_c[P - X0_c + 2]
    // vbar(c) from the view columns c with X0_c - 2 <= P <= X0_c + 3 (X0 grows
    // with c, so they are consecutive: at most 6 / t + 1 of them)
    for (int e = threadIdx.x; e < nrows * T.bw; e += blockDim.x) {
        const int r = e / T.bw, p = e - r * T.bw, Pp_ = T.bx0 + p;
        int lo = 0, hi = ncols;   // first column with X0 + 3 >= P
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (tX0[mid] + 3 >= Pp_) hi = mid; else lo = mid + 1;
        }
        float acc = 0.f;
        for (int c = lo; c < ncols && tX0[c] - 2 <= Pp_; ++c) acc = fmaf(tw[c][Pp_ - tX0[c] + 2], vbs[r][c], acc);
        Bb[r * bw_max + p] = acc;
    }
    // dL/dt through X: sum vbar dv/dX (x - (Wv - 1)/2)
    float tb = 0.f;
    for (int e = threadIdx.x; e < nrows * ncols; e += blockDim.x) {
        const int r = e / ncols, c = e - r * ncols;
        const int X0 = tX0[c];
        const float *Brow = Bs + r * bw_max - T.bx0;
        float dvdX = 0.f;
#pragma unroll
        for (int m = 0; m < 6; ++m) dvdX = fmaf(tdw[c][m], Brow[X0 + m - 2], dvdX);
        tb = fmaf(vbs[r][c] * dvdX, (float)(T.xa + c) - T.crv, tb);
    }
    __syncthreads();

    // strip positions folded onto their (clamped) canvas columns: an inner
    // column is one strip position, the canvas edges sum the clamped ones;
    // the pad columns are zero
    const int bcw = T.cw + 2 * kBcPad;
    for (int e = threadIdx.x; e < nrows * bcw; e += blockDim.x) {
        const int r = e / bcw, c = e - r * bcw - kBcPad, ic = T.clo + c;
        const float *Bbrow = Bb + r * bw_max;
        float acc = 0.f;
        if (c >= 0 && c < T.cw) {
            if (ic > 0 && ic < last) {
                const int p = ic - T.bx0;
                if (p >= 0 && p < T.bw) acc = Bbrow[p];
            } else {
                for (int p = 0; p < T.bw; ++p) acc += (clampi(T.bx0 + p, 0, last) == ic) ? Bbrow[p] : 0.f;
            }
        }
        Bc[r * bcp + kBcPad + c] = acc;
    }
    __syncthreads();

    // Gaussian transposed as a gather: B(ic) = g0 C(ic) + sum_k g_k (C(max(ic-k, 0))
    // + C(min(ic+k, last))), so an inner column col takes g_|ic - col| from each
    // ic within K; the canvas edges 0 and last also take the clamped taps.  The
    // same coefficients with dg/dsigma give dL/dsigma = sum_ic Bbar(ic) dB(ic)/dsigma
    // = sum_col C(col) sum_ic Bbar(ic) dcoef(ic, col).
    float sb = 0.f;
    for (int e = threadIdx.x; e < nrows * T.cw; e += blockDim.x) {
        const int r = e / T.cw, c = e - r * T.cw;
        const int col = T.clo + c;
        const float *Bcrow = Bc + r * bcp + kBcPad - T.clo;
        float acc = 0.f, dacc = 0.f;
        if (col > 0 && col < last) {
            // symmetric taps in pairs; columns beyond clo .. chi read the zero pads
            const float *b = Bcrow + col;
            acc = g[0] * b[0];
            dacc = dg[0] * b[0];
            for (int k = 1; k <= K; ++k) {
                const float pair = b[-k] + b[k];
                acc = fmaf(g[k], pair, acc);
                dacc = fmaf(dg[k], pair, dacc);
            }
        } else {
            for (int ic = max(col - K, T.clo); ic <= min(col + K, T.chi); ++ic) {
                float coef = ic == col ? g[0] : 0.f, dcoef = ic == col ? dg[0] : 0.f;
                for (int k = 1; k <= K; ++k) {
                    const float n = (float)((max(ic - k, 0) == col) + (min(ic + k, last) == col));
                    coef = fmaf(g[k], n, coef);
                    dcoef = fmaf(dg[k], n, dcoef);
                }
                acc = fmaf(coef, Bcrow[ic], acc);
                dacc = fmaf(dcoef, Bcrow[ic], dacc);
            }
        }
        Cb[r * cw_max + c] = acc;
        sb = fmaf(Cs[r * cw_max + c], dacc, sb);
    }
    __syncthreads();

    // rotation transposed: dL/dp -> (phi, tx, ty) from the stored dC/dp
    float pb = 0.f, txb = 0.f, tyb = 0.f, cmax = 0.f;
    const float dg2r = 0.017453292519943295f;
    for (int e = threadIdx.x; e < nrows * T.cw; e += blockDim.x) {
        const int r = e / T.cw, c = e - r * T.cw;
        const int i = T.clo + c;
        const float cb = Cb[r * cw_max + c];
        if (cb == 0.f) continue;
        const int j = T.j0 + r;
        const float dcdx = Cx[r * cw_max + c], dcdy = Cy[r * cw_max + c];
        const float dx = (float)i - G.crx, dy = (float)j - G.cry;
        txb = fmaf(cb, dcdx, txb);
        tyb = fmaf(cb, dcdy, tyb);
        pb = fmaf(cb, dcdx * (-G.s * dx + G.c * dy) + dcdy * (-G.c * dx - G.s * dy), pb);
        cmax = isfinite(cb) ? fmaxf(cmax, fabsf(cb)) : INFINITY;   // non-finite: the float path
    }

    // and, when asked for, u-bar through the rotation's weights: blocks of
    // 32 canvas columns x the tile's rows (one point per thread) add into a
    // shared-memory patch over their taps' source box, which then goes to
    // u-bar with one global atomic per touched pixel (two patches alternate,
    // so one barrier separates a block's adds from its flush).  The patch
    // holds fixed point with scale 2^(24 - k), where 2^k bounds the tile's
    // |C-bar|: a patch pixel sums at most 36 products of at most 1.2 |C-bar|,
    // below 2^31 / scale, and each product is rounded by at most 2^-25 of the
    // tile's largest |C-bar|.
    if (V.ubar) {
        __shared__ int patch[2][kPatch * kPatchPitch];
        const float cm = block_max_all(cmax, red);
        int k2;
        frexpf(cm, &k2);
        const bool fixed = cm >= 1e-30f && cm < INFINITY;
        const float scale = fixed ? ldexpf(1.f, 24 - k2) : 0.f, inv = fixed ? ldexpf(1.f, k2 - 24) : 0.f;
        const int Wu = V.W, Hu = V.H;
        const int r = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31u);
        int buf = 0;
        for (int q0 = 0; q0 < T.cw && cm > 0.f; q0 += 32, buf ^= 1) {
            const int qn = min(32, T.cw - q0);
            int bx0 = INT_MAX, bx1 = INT_MIN, by0 = INT_MAX, by1 = INT_MIN;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float px, py;
                G.map(T.clo + q0 + ((k & 1) ? qn - 1 : 0), T.j0 + ((k & 2) ? nrows - 1 : 0), px, py);
                const int fx = (int)floorf(px), fy = (int)floorf(py);
                bx0 = min(bx0, fx);
                bx1 = max(bx1, fx);
                by0 = min(by0, fy);
                by1 = max(by1, fy);
            }
            // taps floor - 2 .. floor + 3, one pixel more either side for the
            // rounding of the interior points' positions, clamped like the taps
            bx0 = clampi(bx0 - 3, 0, Wu - 1);
            bx1 = clampi(bx1 + 4, 0, Wu - 1);
            by0 = clampi(by0 - 3, 0, Hu - 1);
            by1 = clampi(by1 + 4, 0, Hu - 1);
            const int PW = bx1 - bx0 + 1, PH = by1 - by0 + 1;
            const bool fits = fixed && PW <= kPatch && PH <= kPatch;
            int *P = patch[buf];
            if (fits)
                for (int ly = r; ly < PH; ly += kDThreads / 32)
                    for (int lx = lane; lx < PW; lx += 32) P[ly * kPatchPitch + lx] = 0;
            __syncthreads();
            const int c = q0 + lane;
            if (lane < qn && r < nrows) {
                const float cb = Cb[r * cw_max + c];
                if (cb != 0.f) {
                    float px, py;
                    G.map(T.clo + c, T.j0 + r, px, py);
                    if (fits) scatter_patch(P, bx0, by0, PW, PH, scale, V.ubar, Wu, Hu, px, py, cb);
                    else scatter_ubar(V.ubar, Wu, Hu, px, py, cb);
                }
            }
            __syncthreads();
            if (fits)
                for (int ly = r; ly < PH; ly += kDThreads / 32)
                    for (int lx = lane; lx < PW; lx += 32) {
                        const int v = P[ly * kPatchPitch + lx];
                        if (v != 0) atomicAdd(V.ubar + (size_t)(by0 + ly) * Wu + bx0 + lx, (float)v * inv);
                    }
        }
    }
    const float s_tb = block_sum(tb, red);
    const float s_sb = block_sum(sb, red);
    const float s_pb = block_sum(pb, red);
    const float s_tx = block_sum(txb, red);
    const float s_ty = block_sum(tyb, red);
    if (threadIdx.x == 0) {
        const double dt = (double)s_tb + (double)s_sb * Pp.dsig_dt;
        atomicAdd(V.pbar + 0, dt);
        atomicAdd(V.pbar + 1, (double)s_pb * dg2r);
        atomicAdd(V.pbar + 2, (double)s_tx);
        atomicAdd(V.pbar + 3, (double)s_ty);
    }
}

// ---------------------------------------------------------------- photometric descent
// Per view i (blockIdx.y): loss_i = mean over its pixels of (v - target)^2
// (squares in fp32, sums in fp64) and, when vbar is given, the gradient of
// the summed losses, vbar = 2 (v - target) / count_i.
__global__ void __launch_bounds__(256)
warp_loss_kernel(const WarpSeg *__restrict__ segs, const float *__restrict__ v, const float *__restrict__ target,
                 double *__restrict__ loss, float *__restrict__ vbar)
{
    __shared__ double red[8];
    const WarpSeg S = segs[blockIdx.y];
    const float inv2 = 2.0f / (float)S.count;
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < S.count;
         k += (long long)gridDim.x * blockDim.x) {
        const float d = v[S.off + k] - target[S.off + k];
        acc += (double)(d * d);
        if (vbar) vbar[S.off + k] = inv2 * d;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        atomicAdd(loss + blockIdx.y, t / (double)S.count);
    }
}

// One thread per view: Adam on (t, phi, tx, ty) with step sizes lr scaled by
// decay^step, b1 = 0.9, b2 = 0.999, eps = 1e-12; a view whose gradient is not
// finite takes a zero gradient (its moments still move it); t is clamped to
// [t_lo, t_hi].
__global__ void __launch_bounds__(128)
warp_adam_kernel(int n, double *__restrict__ params, const double *__restrict__ grad, double *__restrict__ m,
                 double *__restrict__ v, const AdamArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool finite = true;
    double g[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        g[k] = grad[4 * i + k];
        finite &= isfinite(g[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double gk = finite ? g[k] : 0.0;
        const double mk = 0.9 * m[4 * i + k] + 0.1 * gk;
        const double vk = 0.999 * v[4 * i + k] + 0.001 * gk * gk;
        m[4 * i + k] = mk;
        v[4 * i + k] = vk;
        double p = params[4 * i + k] - a.scale * a.lr[k] * (mk / a.c1) / (sqrt(vk / a.c2) + 1e-12);
        if (k == 0) p = fmin(fmax(p, a.t_lo), a.t_hi);
        params[4 * i + k] = p;
    }
}

// ---------------------------------------------------------------- host side
int dwarp_tile_width(bool backward) { return backward ? kDTWBwd : kDTWFwd; }

void dwarp_strip_widths(int tw, double t_max, int K, int *cw, int *bw)
{
    const int span = (int)std::ceil(t_max * (tw - 1)) + 2;
    *bw = span + 6;
    *cw = *bw + 2 * K;
}

int dwarp_tiles(int Wv, int Hv, int tw, int *ntx)
{
    *ntx = (Wv + tw - 1) / tw;
    return *ntx * ((Hv + kDTH - 1) / kDTH);
}

cudaError_t launch_dwarp(bool backward, const DiffView *d_views, DiffPrep *d_prep, int n_views, int n_tiles,
                         int cw_max, int bw_max, int32_t *status, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    dwarp_prep_kernel<<<n_views, 64, 0, s>>>(d_views, d_prep);
    note_launch();
    const size_t smem =
        sizeof(float) * (size_t)kDTH * (backward ? 5 * cw_max + 2 * kBcPad + 2 * bw_max : cw_max + bw_max);
    if (backward) {
        const cudaError_t e = ensure_dynamic_smem((const void *)dwarp_bwd_kernel, smem);
        if (e != cudaSuccess) return e;
        dwarp_bwd_kernel<<<n_tiles, kDThreads, smem, s>>>(d_views, d_prep, n_views, cw_max, bw_max, status);
    } else {
        const cudaError_t e = ensure_dynamic_smem((const void *)dwarp_fwd_kernel, smem);
        if (e != cudaSuccess) return e;
        dwarp_fwd_kernel<<<n_tiles, kDThreads, smem, s>>>(d_views, d_prep, n_views, cw_max, bw_max, status);
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_warp_loss(const WarpSeg *d_segs, int n, long long max_count, const float *v, const float *target,
                             double *loss, float *vbar, cudaStream_t s)
{
    if (n <= 0 || max_count <= 0) return cudaSuccess;
    const int bx = (int)std::min<long long>((max_count + 255) / 256, 64);
    warp_loss_kernel<<<dim3(bx, n), 256, 0, s>>>(d_segs, v, target, loss, vbar);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_warp_adam(int n, double *params, const double *grad, double *m, double *v, const AdamArgs &a,
                             cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    warp_adam_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, params, grad, m, v, a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asift
