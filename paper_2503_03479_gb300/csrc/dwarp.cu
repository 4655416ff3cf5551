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
// is accumulated with shared-memory atomics, folded onto canvas columns, and
// C-bar (the Gaussian transposed) gathered from it; C-bar drives the
// parameter derivatives through the stored dC/dp and, when the image gradient
// is asked for, scatters into u-bar (the rotation transposed) with global
// atomics.  Tiles only add partial adjoints, so the sum over tiles is the
// exact transpose (up to fp32 summation order).
#include "common.cuh"
#include "kernels.h"

namespace asift {

constexpr int kDTW = 32, kDTH = 8, kDThreads = 256;

// sinc and its derivative; series below |x| < 1e-2 where the closed forms cancel.
__device__ __forceinline__ void sinc_d(float x, float &sc, float &dsc)
{
    const float ax = fabsf(x);
    if (ax < 1e-2f) {
        const float y = 9.8696044010893586f * x * x;   // (pi x)^2
        sc = 1.f - y * (1.f / 6.f) * (1.f - y * (1.f / 20.f));
        dsc = -3.2898681336964529f * x * (1.f - y * (1.f / 10.f));   // -(pi^2 x / 3)(1 - (pi x)^2/10)
        return;
    }
    float s, c;
    sincospif(x, &s, &c);
    sc = s / (3.14159265358979f * x);
    dsc = (c - sc) / x;
}

// Normalised Lanczos-3 weights w_m(f) (m = -2..3) and dw_m/df from L and L'
// evaluated tap by tap (L' is needed for the backward; the forward uses the
// same evaluation so both see one function).
__device__ __forceinline__ void lanczos3_wd(float f, float w[6], float dw[6])
{
    float L[6], dL[6], S = 0.f, dS = 0.f;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const float x = f - (float)(m - 2);
        if (fabsf(x) < 3.f) {
            float a, da, b, db;
            sinc_d(x, a, da);
            sinc_d(x * (1.f / 3.f), b, db);
            L[m] = a * b;
            dL[m] = da * b + a * db * (1.f / 3.f);
        } else {
            L[m] = 0.f;
            dL[m] = 0.f;
        }
        S += L[m];
        dS += dL[m];
    }
    const float inv = 1.f / S;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        w[m] = L[m] * inv;
        dw[m] = (dL[m] - w[m] * dS) * inv;
    }
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

// Canvas value at p, optionally with dC/dpx, dC/dpy, and optionally
// scattering cb * w_x w_y into ubar.
__device__ __forceinline__ float canvas_at(const float *__restrict__ u, int W, int H, float px, float py,
                                           float *dcdx, float *dcdy, float cb, float *__restrict__ ubar)
{
    const float fx0 = floorf(px), fy0 = floorf(py);
    const int x0 = (int)fx0, y0 = (int)fy0;
    float wx[6], dwx[6], wy[6], dwy[6];
    lanczos3_wd(px - fx0, wx, dwx);
    lanczos3_wd(py - fy0, wy, dwy);
    int xs[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) xs[m] = clampi(x0 + m - 2, 0, W - 1);
    float acc = 0.f, ax = 0.f, ay = 0.f;
#pragma unroll
    for (int n = 0; n < 6; ++n) {
        const int yy = clampi(y0 + n - 2, 0, H - 1);
        const float *row = u + (size_t)yy * W;
        float r = 0.f, dr = 0.f;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const float val = __ldg(row + xs[m]);
            r = fmaf(wx[m], val, r);
            dr = fmaf(dwx[m], val, dr);
            if (ubar) atomicAdd(ubar + (size_t)yy * W + xs[m], cb * wx[m] * wy[n]);
        }
        acc = fmaf(wy[n], r, acc);
        ax = fmaf(wy[n], dr, ax);
        ay = fmaf(dwy[n], r, ay);
    }
    if (dcdx) *dcdx = ax;
    if (dcdy) *dcdy = ay;
    return acc;
}

__device__ __forceinline__ float sigma_of(double t) { return t > 1.0 ? (float)(0.8 * sqrt(t * t - 1.0)) : 0.f; }

// Gaussian taps g_0..g_K (and dg/dsigma) into shared memory.
__device__ void gauss_taps(float sigma, int K, float *g, float *dg)
{
    __shared__ float E, M2;
    if (threadIdx.x == 0) {
        float e = 0.f, m2 = 0.f;
        if (sigma > 0.f) {
            for (int k = 0; k <= K; ++k) {
                const float v = expf(-(float)(k * k) / (2.f * sigma * sigma));
                e += (k == 0) ? v : 2.f * v;
            }
            for (int k = 1; k <= K; ++k) m2 += 2.f * expf(-(float)(k * k) / (2.f * sigma * sigma)) * (float)(k * k);
            m2 /= e;
        }
        E = e;
        M2 = m2;
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= K; k += blockDim.x) {
        if (sigma > 0.f) {
            g[k] = expf(-(float)(k * k) / (2.f * sigma * sigma)) / E;
            dg[k] = g[k] * ((float)(k * k) - M2) / (sigma * sigma * sigma);
        } else {
            g[k] = (k == 0) ? 1.f : 0.f;
            dg[k] = 0.f;
        }
    }
    __syncthreads();
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
    T.xa = tx * kDTW;
    T.xb = min(T.xa + kDTW, V.Wv) - 1;
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

__device__ __forceinline__ DGeom dgeom(const DiffView &V)
{
    const double r = V.param[1] * (3.14159265358979323846 / 180.0);
    DGeom G;
    G.c = (float)cos(r);
    G.s = (float)sin(r);
    G.cx = (V.W - 1) * 0.5f;
    G.cy = (V.H - 1) * 0.5f;
    G.tx = (float)V.param[2];
    G.ty = (float)V.param[3];
    G.crx = (V.Wr - 1) * 0.5f;
    G.cry = (V.Hr - 1) * 0.5f;
    return G;
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
            Cs[r * cw_max + c] = canvas_at(V.u, V.W, V.H, px, py, &dx, &dy, 0.f, nullptr);
            Cx[r * cw_max + c] = dx;
            Cy[r * cw_max + c] = dy;
        } else {
            Cs[r * cw_max + c] = canvas_at(V.u, V.W, V.H, px, py, nullptr, nullptr, 0.f, nullptr);
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
dwarp_fwd_kernel(const DiffView *__restrict__ views, int n_views, int cw_max, int bw_max, int32_t *status)
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
    const DGeom G = dgeom(V);
    gauss_taps(sigma_of(V.param[0]), V.K, g, dg);
    strips(V, T, G, g, Cs, Bs, cw_max, bw_max);
    const int nrows = T.j1 - T.j0 + 1, ncols = T.xb - T.xa + 1;
    const float cr = (V.Wr - 1) * 0.5f;
    for (int e = threadIdx.x; e < nrows * ncols; e += blockDim.x) {
        const int r = e / ncols, c = e - r * ncols;
        const int x = T.xa + c;
        const float X = T.t * ((float)x - T.crv) + cr;
        const float fX = floorf(X);
        const int X0 = (int)fX;
        float w[6], dw[6];
        lanczos3_wd(X - fX, w, dw);
        const float *Brow = Bs + r * bw_max - T.bx0;
        float v = 0.f;
#pragma unroll
        for (int m = 0; m < 6; ++m) v = fmaf(w[m], Brow[X0 + m - 2], v);
        V.out[(size_t)(T.j0 + r) * V.Wv + x] = v;
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
dwarp_bwd_kernel(const DiffView *__restrict__ views, int n_views, int cw_max, int bw_max, int32_t *status)
{
    extern __shared__ float sm[];
    float *Cs = sm, *Cx = Cs + kDTH * cw_max, *Cy = Cx + kDTH * cw_max, *Cb = Cy + kDTH * cw_max;
    float *Bc = Cb + kDTH * cw_max;                  // B-bar folded onto canvas columns (clo .. chi)
    float *Bs = Bc + kDTH * cw_max, *Bb = Bs + kDTH * bw_max;
    __shared__ float g[ASIFT_MAX_GAUSS], dg[ASIFT_MAX_GAUSS], red[kDThreads / 32];
    const DTile T = dtile(views, n_views, blockIdx.x);
    const DiffView &V = views[T.v];
    if (T.cw > cw_max || T.bw > bw_max || V.K >= ASIFT_MAX_GAUSS) {
        if (threadIdx.x == 0) set_status(status, ASIFT_ERR_CAPACITY);
        return;
    }
    const DGeom G = dgeom(V);
    const float sigma = sigma_of(V.param[0]);
    const int K = V.K, last = V.Wr - 1;
    gauss_taps(sigma, K, g, dg);
    strips(V, T, G, g, Cs, Bs, cw_max, bw_max, Cx, Cy);
    const int nrows = T.j1 - T.j0 + 1, ncols = T.xb - T.xa + 1;
    for (int e = threadIdx.x; e < kDTH * bw_max; e += blockDim.x) Bb[e] = 0.f;
    for (int e = threadIdx.x; e < kDTH * cw_max; e += blockDim.x) Bc[e] = 0.f;
    __syncthreads();

    // tilt transposed: B-bar at the strip positions (six shared atomics per
    // view pixel), and dL/dt through X
    const float cr = (V.Wr - 1) * 0.5f;
    float tb = 0.f;
    for (int e = threadIdx.x; e < nrows * ncols; e += blockDim.x) {
        const int r = e / ncols, c = e - r * ncols;
        const int x = T.xa + c;
        const float vb = V.vbar[(size_t)(T.j0 + r) * V.Wv + x];
        const float X = T.t * ((float)x - T.crv) + cr;
        const float fX = floorf(X);
        const int X0 = (int)fX;
        float w[6], dw[6];
        lanczos3_wd(X - fX, w, dw);
        const float *Brow = Bs + r * bw_max - T.bx0;
        float *Bbrow = Bb + r * bw_max - T.bx0;
        float dvdX = 0.f;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            // strip position X0+m-2 holds column clamp(X0+m-2): the clamped
            // taps of the forward accumulate at their strip positions
            atomicAdd(Bbrow + X0 + m - 2, w[m] * vb);
            dvdX = fmaf(dw[m], Brow[X0 + m - 2], dvdX);
        }
        tb = fmaf(vb * dvdX, (float)x - T.crv, tb);
    }
    __syncthreads();

    // strip positions folded onto their (clamped) canvas columns, and dL/dsigma
    float sb = 0.f;
    for (int e = threadIdx.x; e < nrows * T.bw; e += blockDim.x) {
        const int r = e / T.bw, c = e - r * T.bw;
        const float b = Bb[r * bw_max + c];
        if (b == 0.f) continue;
        const int ic = clampi(T.bx0 + c, 0, last);
        atomicAdd(Bc + r * cw_max + ic - T.clo, b);
        const float *Crow = Cs + r * cw_max - T.clo;
        float ds = dg[0] * Crow[ic];
        for (int k = 1; k <= K; ++k) ds = fmaf(dg[k], Crow[max(ic - k, 0)] + Crow[min(ic + k, last)], ds);
        sb = fmaf(b, ds, sb);
    }
    __syncthreads();

    // Gaussian transposed as a gather: B(ic) = g0 C(ic) + sum_k g_k (C(max(ic-k, 0))
    // + C(min(ic+k, last))), so an inner column col takes g_|ic - col| from each
    // ic within K; the canvas edges 0 and last also take the clamped taps
    for (int e = threadIdx.x; e < nrows * T.cw; e += blockDim.x) {
        const int r = e / T.cw, c = e - r * T.cw;
        const int col = T.clo + c;
        const float *Bcrow = Bc + r * cw_max - T.clo;
        float acc = 0.f;
        if (col > 0 && col < last) {
            const int lo = max(col - K, T.clo), hi = min(col + K, T.chi);
            for (int ic = lo; ic <= hi; ++ic) acc = fmaf(g[abs(ic - col)], Bcrow[ic], acc);
        } else {
            for (int ic = max(col - K, T.clo); ic <= min(col + K, T.chi); ++ic) {
                float coef = ic == col ? g[0] : 0.f;
                for (int k = 1; k <= K; ++k)
                    coef += g[k] * (float)((max(ic - k, 0) == col) + (min(ic + k, last) == col));
                acc = fmaf(coef, Bcrow[ic], acc);
            }
        }
        Cb[r * cw_max + c] = acc;
    }
    __syncthreads();

    // rotation transposed: dL/dp -> (phi, tx, ty) from the stored dC/dp, and
    // (when asked for) u-bar by scattering through the rotation's weights
    float pb = 0.f, txb = 0.f, tyb = 0.f;
    const float dg2r = 0.017453292519943295f;
    for (int e = threadIdx.x; e < nrows * T.cw; e += blockDim.x) {
        const int r = e / T.cw, c = e - r * T.cw;
        const int i = T.clo + c;
        const float cb = Cb[r * cw_max + c];
        if (cb == 0.f) continue;
        const int j = T.j0 + r;
        const float dcdx = Cx[r * cw_max + c], dcdy = Cy[r * cw_max + c];
        if (V.ubar) {
            float px, py;
            G.map(i, j, px, py);
            canvas_at(V.u, V.W, V.H, px, py, nullptr, nullptr, cb, V.ubar);
        }
        const float dx = (float)i - G.crx, dy = (float)j - G.cry;
        txb = fmaf(cb, dcdx, txb);
        tyb = fmaf(cb, dcdy, tyb);
        pb = fmaf(cb, dcdx * (-G.s * dx + G.c * dy) + dcdy * (-G.c * dx - G.s * dy), pb);
    }
    const float s_tb = block_sum(tb, red);
    const float s_sb = block_sum(sb, red);
    const float s_pb = block_sum(pb, red);
    const float s_tx = block_sum(txb, red);
    const float s_ty = block_sum(tyb, red);
    if (threadIdx.x == 0) {
        const double t = V.param[0];
        double dt = s_tb;
        if (t > 1.0) dt += (double)s_sb * 0.8 * t / sqrt(t * t - 1.0);
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
void dwarp_strip_widths(int Wv, double t_max, int K, int *cw, int *bw)
{
    (void)Wv;
    const int span = (int)std::ceil(t_max * (kDTW - 1)) + 2;
    *bw = span + 6;
    *cw = *bw + 2 * K;
}

int dwarp_tiles(int Wv, int Hv, int *ntx)
{
    *ntx = (Wv + kDTW - 1) / kDTW;
    return *ntx * ((Hv + kDTH - 1) / kDTH);
}

cudaError_t launch_dwarp(bool backward, const DiffView *d_views, int n_views, int n_tiles, int cw_max, int bw_max,
                         int32_t *status, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * (size_t)kDTH * (backward ? 5 * cw_max + 2 * bw_max : cw_max + bw_max);
    if (backward) {
        const cudaError_t e = ensure_dynamic_smem((const void *)dwarp_bwd_kernel, smem);
        if (e != cudaSuccess) return e;
        dwarp_bwd_kernel<<<n_tiles, kDThreads, smem, s>>>(d_views, n_views, cw_max, bw_max, status);
    } else {
        const cudaError_t e = ensure_dynamic_smem((const void *)dwarp_fwd_kernel, smem);
        if (e != cudaSuccess) return e;
        dwarp_fwd_kernel<<<n_tiles, kDThreads, smem, s>>>(d_views, n_views, cw_max, bw_max, status);
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
