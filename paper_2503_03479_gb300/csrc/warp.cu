// warp.cu -- affine view simulation (Eq. (2)-(4)) on sm_103a.
//
// One CTA produces a tw x kWarpTH tile of one view (tw <= kWarpTW chosen per
// view, see warp_tile_width).  A view row j only depends on canvas row j (the
// tilt acts along canvas x), so the tile needs a canvas strip of kWarpTH rows
// and columns [bx0 - K, bx1 + K], where [bx0, bx1] = [floor(X(x'_first)) - 2,
// floor(X(x'_last)) + 3] are the columns the tilt taps read.  The CTA:
//   1. computes the rotated canvas C on that strip in chunks of kChunk
//      columns; for each chunk the source pixels its 6x6 Lanczos-3 taps can
//      reach (the bounding box of the rotated chunk, at most 41 x 44, rounded
//      out to 16-byte groups) are staged in shared memory with asynchronous
//      copies, double-buffered, so every tap is a shared-memory load
//      (Eq. (3)-(4); geometry in exact Q32 fixed point);
//   2. applies the Gaussian along x and the Lanczos-3 tilt resampling at
//      X = t (x' - (Wv-1)/2) + (Wr-1)/2 as one filter per view column
//      (computed once per view by tilt_filter_kernel), and writes fp32
//      (optional), rint-to-u8 and the footprint mask.
// Strip position i holds the value of canvas column clamp(i, 0, Wr-1), which
// realises the clamped borders of the Gaussian and of the tilt taps without
// per-tap clamps.
// Every launch covers a list of views (one view for the per-view form, all
// views of several images for the batched form); a CTA finds its view by a
// warp-wide search over the views' first tile index.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace asift {

constexpr int kChunk = 32;              // canvas columns per staged chunk
constexpr int kStage = 41;              // staged source box (rows), >= 32|c| + 16|s| + 6
constexpr int kPitchMin = 44, kPitchMax = 48;   // row pitch of the staged box (44 or 48), chosen per view
constexpr int kStageBuf = kStage * kPitchMax;   // floats per staging buffer (two, double-buffered)

// The hardware reciprocal (rcp.approx: relative error within one ulp).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

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
//   w_m  ~  N_m / D_m,  N_m = (-1)^m sin(pi f/3 - pi m/3),  D_m = (f - m)^2,
// whose six sines follow from sin and cos of pi f/3 by angle addition.  Over
// the common denominator, w_m = N_m prod_{k != m} D_k / sum_n N_n prod_{k != n}
// D_k: prefix and suffix products and one reciprocal.  f is the top 23
// fraction bits (an error below 1.2e-7 px); f = 0 there is the identity.
__device__ __forceinline__ void lanczos3_weights(uint32_t lo, float w[6])
{
    const uint32_t m23 = lo >> 9;
    if (m23 == 0u) {
        w[0] = w[1] = w[3] = w[4] = w[5] = 0.f;
        w[2] = 1.f;
        return;
    }
    const float f = __uint_as_float(0x3F800000u | m23) - 1.0f;   // exact: m23 * 2^-23
    float s, c;
    sincos_small(f * 1.04719755119659775f, s, c);
    const float hs = 0.5f * s, hc = 0.86602540378443864676f * c;
    const float a = hc - hs, b = -(hs + hc);
    const float d0 = f + 2.f, d1 = f + 1.f, d3 = f - 1.f, d4 = f - 2.f, d5 = f - 3.f;
    const float D0 = d0 * d0, D1 = d1 * d1, D2 = f * f, D3 = d3 * d3, D4 = d4 * d4, D5 = d5 * d5;
    const float p2 = D0 * D1, p3 = p2 * D2, p4 = p3 * D3;           // prefix products
    const float s3 = D5 * D4, s2 = s3 * D3, s1 = s2 * D2;           // suffix products
    const float u0 = a * (s1 * D1), u1 = b * (D0 * s1), u2 = s * (p2 * s2);
    const float u3 = a * (p3 * s3), u4 = b * (p4 * D5), u5 = s * (p4 * D4);
    const float inv = __frcp_rn(((u0 + u1) + (u2 + u3)) + (u4 + u5));
    w[0] = u0 * inv; w[1] = u1 * inv; w[2] = u2 * inv;
    w[3] = u3 * inv; w[4] = u4 * inv; w[5] = u5 * inv;
}

// Two weight sets at once in packed fp32 pairs (.x from lo_a, .y from lo_b),
// the same arithmetic as lanczos3_weights component by component.  A zero fraction is
// computed at 2^-23 (finite) and then replaced by the exact identity.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

__device__ __forceinline__ void lanczos3_weights2(uint32_t lo_a, uint32_t lo_b, float2 w[6])
{
    const uint32_t ma = lo_a >> 9, mb = lo_b >> 9;
    const float2 f = make_float2(__uint_as_float(0x3F800000u | max(ma, 1u)) - 1.0f,
                                 __uint_as_float(0x3F800000u | max(mb, 1u)) - 1.0f);
    const float2 x = __fmul2_rn(f, f2(1.04719755119659775f));
    const float2 x2 = __fmul2_rn(x, x);
    float2 ps = __ffma2_rn(x2, f2(2.75573192e-6f), f2(-1.98412698e-4f));
    ps = __ffma2_rn(x2, ps, f2(8.33333333e-3f));
    ps = __ffma2_rn(x2, ps, f2(-1.66666667e-1f));
    ps = __ffma2_rn(x2, ps, f2(1.0f));
    const float2 s = __fmul2_rn(x, ps);
    float2 pc = __ffma2_rn(x2, f2(-2.75573192e-7f), f2(2.48015873e-5f));
    pc = __ffma2_rn(x2, pc, f2(-1.38888889e-3f));
    pc = __ffma2_rn(x2, pc, f2(4.16666667e-2f));
    pc = __ffma2_rn(x2, pc, f2(-0.5f));
    const float2 c = __ffma2_rn(x2, pc, f2(1.0f));
    const float2 hs = __fmul2_rn(f2(0.5f), s), hc = __fmul2_rn(f2(0.86602540378443864676f), c);
    const float2 a = __fadd2_rn(hc, __fmul2_rn(hs, f2(-1.0f)));
    const float2 b = __fmul2_rn(__fadd2_rn(hs, hc), f2(-1.0f));
    const float2 d0 = __fadd2_rn(f, f2(2.f)), d1 = __fadd2_rn(f, f2(1.f)), d3 = __fadd2_rn(f, f2(-1.f));
    const float2 d4 = __fadd2_rn(f, f2(-2.f)), d5 = __fadd2_rn(f, f2(-3.f));
    const float2 D0 = __fmul2_rn(d0, d0), D1 = __fmul2_rn(d1, d1), D2 = __fmul2_rn(f, f);
    const float2 D3 = __fmul2_rn(d3, d3), D4 = __fmul2_rn(d4, d4), D5 = __fmul2_rn(d5, d5);
    const float2 p2 = __fmul2_rn(D0, D1), p3 = __fmul2_rn(p2, D2), p4 = __fmul2_rn(p3, D3);
    const float2 s3 = __fmul2_rn(D5, D4), s2 = __fmul2_rn(s3, D3), s1 = __fmul2_rn(s2, D2);
    const float2 u0 = __fmul2_rn(a, __fmul2_rn(s1, D1)), u1 = __fmul2_rn(b, __fmul2_rn(D0, s1));
    const float2 u2 = __fmul2_rn(s, __fmul2_rn(p2, s2)), u3 = __fmul2_rn(a, __fmul2_rn(p3, s3));
    const float2 u4 = __fmul2_rn(b, __fmul2_rn(p4, D5)), u5 = __fmul2_rn(s, __fmul2_rn(p4, D4));
    const float2 sum = __fadd2_rn(__fadd2_rn(__fadd2_rn(u0, u1), __fadd2_rn(u2, u3)), __fadd2_rn(u4, u5));
    const float2 inv = make_float2(rcp_approx(sum.x), rcp_approx(sum.y));   // within 1 ulp: far below the warp's tolerance
    w[0] = __fmul2_rn(u0, inv); w[1] = __fmul2_rn(u1, inv); w[2] = __fmul2_rn(u2, inv);
    w[3] = __fmul2_rn(u3, inv); w[4] = __fmul2_rn(u4, inv); w[5] = __fmul2_rn(u5, inv);
    if (ma == 0u || mb == 0u) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            if (ma == 0u) w[m].x = m == 2 ? 1.f : 0.f;
            if (mb == 0u) w[m].y = m == 2 ? 1.f : 0.f;
        }
    }
}

// dst: H rows of dpitch floats; the columns from W on are written as zeros.
__global__ void u8_to_f32_kernel(const uint8_t *__restrict__ src, int pitch, int W, int H,
                                 float *__restrict__ dst, int dpitch)
{
    const long long n = (long long)dpitch * H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / dpitch), x = (int)(i - (long long)y * dpitch);
        dst[i] = x < W ? (float)src[(size_t)y * pitch + x] : 0.f;
    }
}

// Every image of a list: blockIdx.y selects the image, x strides its pixels.
__global__ void convert_images_kernel(const ImageConv *__restrict__ list)
{
    const ImageConv c = list[blockIdx.y];
    const long long n = (long long)c.dpitch * c.H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / c.dpitch), x = (int)(i - (long long)y * c.dpitch);
        c.dst[i] = x < c.W ? (float)c.src[(size_t)y * c.pitch + x] : 0.f;
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

// The 36-tap interpolation of the staged source at the Q32 point (px, py),
// all taps inside the staged box; the x and y weight sets are computed
// together in packed fp32 pairs.
__device__ __forceinline__ float interp_interior(const float *__restrict__ Ss, int P, long long px, long long py,
                                                 int sx0, int sy0)
{
    float2 w[6];
    lanczos3_weights2((uint32_t)px, (uint32_t)py, w);
    const float *b = Ss + ((int)(py >> 32) - 2 - sy0) * P + ((int)(px >> 32) - 2 - sx0);
    // rows (0, 1), (2, 3), (4, 5) as packed pairs: one FFMA2 per column and pair,
    // then the vertical weights as three more
    float2 a01, a23, a45;
    {
        const float2 wx = make_float2(w[0].x, w[0].x);
        a01 = __fmul2_rn(wx, make_float2(b[0], b[P]));
        a23 = __fmul2_rn(wx, make_float2(b[2 * P], b[3 * P]));
        a45 = __fmul2_rn(wx, make_float2(b[4 * P], b[5 * P]));
    }
#pragma unroll
    for (int m = 1; m < 6; ++m) {
        const float2 wx = make_float2(w[m].x, w[m].x);
        a01 = __ffma2_rn(wx, make_float2(b[m], b[P + m]), a01);
        a23 = __ffma2_rn(wx, make_float2(b[2 * P + m], b[3 * P + m]), a23);
        a45 = __ffma2_rn(wx, make_float2(b[4 * P + m], b[5 * P + m]), a45);
    }
    float2 t = __fmul2_rn(make_float2(w[0].y, w[1].y), a01);
    t = __ffma2_rn(make_float2(w[2].y, w[3].y), a23, t);
    t = __ffma2_rn(make_float2(w[4].y, w[5].y), a45, t);
    return t.x + t.y;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Source box of one chunk of the canvas strip: the taps of the four corners
// of the (clamped) canvas region, clamped to the image.  interior: every tap
// of every point of the chunk lies inside the image (the points lie in the
// corners' convex hull), so no clamps and no background test are needed.
// outside: every point lies outside [-1/2, W-1/2) x [-1/2, H-1/2) (all four
// corners beyond one edge), so the chunk is background.  Lanes 0..3 of each
// warp map one corner each and the warp reduces them with shuffles.
struct StageBox {
    int sx0, sy0, bwid, bhgt;
    bool interior, outside;
};

__device__ __forceinline__ StageBox chunk_box(const CanvasGeom &G, int i_lo, int i_hi, int j0, int j1, int W, int H,
                                              unsigned lane)
{
    const int q = lane & 3;
    long long px, py;
    G.map(q & 1 ? i_hi : i_lo, q & 2 ? j1 : j0, px, py);
    int fx = (int)(px >> 32), fy = (int)(py >> 32);
    const long long HALF = 2147483648LL;
    unsigned side = (px < -HALF ? 1u : 0u) | (px >= (long long)(2 * W - 1) * HALF ? 2u : 0u) |
                    (py < -HALF ? 4u : 0u) | (py >= (long long)(2 * H - 1) * HALF ? 8u : 0u);
    int sx0 = fx, sx1 = fx, sy0 = fy, sy1 = fy;
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        sx0 = min(sx0, __shfl_xor_sync(0xffffffffu, sx0, o));
        sx1 = max(sx1, __shfl_xor_sync(0xffffffffu, sx1, o));
        sy0 = min(sy0, __shfl_xor_sync(0xffffffffu, sy0, o));
        sy1 = max(sy1, __shfl_xor_sync(0xffffffffu, sy1, o));
        side &= __shfl_xor_sync(0xffffffffu, side, o);
    }
    StageBox b;
    b.interior = sx0 >= 2 && sx1 + 3 <= W - 1 && sy0 >= 2 && sy1 + 3 <= H - 1;
    b.outside = side != 0u;
    // columns rounded out to whole 16-byte groups of the source rows (pitch a
    // multiple of 4 floats, columns >= W of the last group zero)
    b.sx0 = clampi(sx0 - 2, 0, W - 1) & ~3;
    b.sy0 = clampi(sy0 - 2, 0, H - 1);
    // a chunk spans at most 31 columns and 15 rows of the canvas, so its
    // corners' integer parts differ by at most sqrt(31^2 + 15^2) + 1 < 36 and
    // the box spans at most 35 + 6 = 41 = kStage rows and 35 + 9 = 44 =
    // kPitchMin columns once rounded out to 16-byte groups
    b.bwid = ((clampi(sx1 + 3, 0, W - 1) - b.sx0 + 1) + 3) & ~3;
    b.bhgt = clampi(sy1 + 3, 0, H - 1) - b.sy0 + 1;
    return b;
}

__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// Issues the asynchronous copies of a box into a staging buffer (pitch P, a
// multiple of 4): 16-byte groups, the box's (row, group) pairs dealt out to
// the block's threads in order (thread t takes t, t + 256, ...).
__device__ __forceinline__ void stage_box(float *dst, int P, const float *__restrict__ src, int sp, const StageBox &b,
                                          unsigned warp, unsigned lane)
{
    if (b.outside) return;
    const int nf4 = b.bwid >> 2, tot = b.bhgt * nf4;
    const int t = (int)(warp * 32u + lane);
    // integer quotients by nf4 <= 19 through a float reciprocal: (n + 1/2) / nf4
    // stays 1/38 away from an integer, far above the product's rounding error
    const float inv = __fdividef(1.0f, (float)nf4);
    const int dr = __float2int_rz((kWarpThreads + 0.5f) * inv), dc = kWarpThreads - dr * nf4;   // stride in (row, group)
    int r = __float2int_rz(((float)t + 0.5f) * inv), g = t - r * nf4;
    const float *sbase = src + (size_t)b.sy0 * sp + b.sx0;
    const uint32_t dbase = (uint32_t)__cvta_generic_to_shared(dst);
    for (int el = t; el < tot; el += kWarpThreads) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dbase + 4u * (uint32_t)(r * P + 4 * g)),
                     "l"(sbase + (size_t)r * sp + 4 * g)
                     : "memory");
        r += dr;
        g += dc;
        if (g >= nf4) {
            g -= nf4;
            ++r;
        }
    }
}

constexpr int kMaxChunks = 40;          // chunks of a tile's canvas strip: (seg_w + 2 hK) / kChunk, seg_w <= 1024

// The first view column x in [lo, hi) whose tilt tap base max(floor(X(x)), 0)
// is at least c (hi if none): X(x) = tq (2x - Wv + 1) + (Wr - 1) 2^31 grows with x.
__device__ __forceinline__ int first_col_at(const DevView &V, int c, int lo, int hi)
{
    const long long xoff = (long long)(V.Wr - 1) * 2147483648LL;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const long long X = V.tq * (2LL * mid - V.Wv + 1) + xoff;
        if (max((int)(X >> 32), 0) >= c) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// One tile: canvas rows [j0, j0 + kWarpTH) of a rotation group over the
// canvas columns [c0, c1) of segment `seg`, then every member view's columns
// whose tilt taps start in [c0, c1) (max(floor(X), 0) in [c0, c1)).
__device__ __forceinline__ void warp_band_tile(int tile, const DevRotGroup *__restrict__ groups, int n_groups,
                                               const DevView *__restrict__ views, int seg_w, int cwp,
                                               uint8_t *__restrict__ out_u8, uint8_t *__restrict__ out_mask,
                                               float *__restrict__ out_f32)
{
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    // Cs [kWarpTH][cwp] canvas strip (odd row pitch), then the two staging
    // buffers [kStage][pitch] of step 1 (the members' filters in step 2),
    // then the source boxes of the strip's chunks.
    float *Cs = smem;
    float *Sbuf = Cs + kWarpTH * cwp;
    StageBox *Bx = reinterpret_cast<StageBox *>(Sbuf + 2 * kStageBuf);

    const int gi = find_owner(groups, n_groups, tile, [](const DevRotGroup &g) { return g.tile_start; });
    const DevRotGroup &G = groups[gi];
    const int lt = tile - G.tile_start;
    const int band = lt / G.nseg, seg = lt - band * G.nseg;
    const int Wr = G.Wr, W = G.W, H = G.H, hK = G.hK;
    const int j0 = band * kWarpTH, j1 = min(j0 + kWarpTH, G.Hr) - 1;
    const int nrows = j1 - j0 + 1;
    const int c0 = seg * seg_w, c1 = min(c0 + seg_w, Wr);
    const int cx0 = c0 - hK;                // strip position 0 = canvas column cx0 (clamped)
    const int cw = (c1 - c0) + 2 * hK;
    const int nch = (cw + kChunk - 1) / kChunk;
    const long long HALF = 2147483648LL;
    const CanvasGeom Gm{G.cq, G.sq, (long long)(W - 1) * HALF, (long long)(H - 1) * HALF, Wr, G.Hr};
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    constexpr int kRowStep = kWarpThreads / kChunk;   // step 1: a thread walks its column in steps of kRowStep rows
    constexpr int kFiltStep = 4;                      // step 2: a thread's rows rg, rg + 4, rg + 8, rg + 12
    static_assert(kWarpTH == 4 * kFiltStep, "step 2 keeps four rows per thread");

    // each member's view columns [xa, xb) for step 2, found once per tile by
    // two threads per member (visible after step 1's last barrier)
    __shared__ int mcols[2 * kGroupMax];
    if ((int)threadIdx.x < 2 * G.n_views) {
        const DevView &V = views[G.view[threadIdx.x >> 1]];
        mcols[threadIdx.x] = (threadIdx.x & 1u) == 0u ? first_col_at(V, c0, 0, V.Wv)
                                                      : (c1 >= Wr ? V.Wv : first_col_at(V, c1, 0, V.Wv));
    }

    // 1. the rotated canvas on the strip (strip position i holds canvas
    //    column clamp(cx0 + i, 0, Wr - 1), which realises the clamped borders
    //    of the Gaussian and of the tilt taps without per-tap clamps)
    if (G.identity) {
        // phi = 0, s = 1: every canvas point is a source pixel with zero
        // fraction, where the normalised weights are the identity, so C is
        // the source itself, copied exactly
        const float *__restrict__ src = G.src;
        for (int el = (int)threadIdx.x; el < nrows * cw; el += kWarpThreads) {
            const int r = el / cw, i = el - r * cw;
            Cs[r * cwp + i] = __ldg(src + (size_t)(j0 + r) * G.src_pitch + clampi(cx0 + i, 0, W - 1));
        }
        for (int k = (int)threadIdx.x; k < nch; k += kWarpThreads) {
            StageBox b{};
            b.interior = true;
            b.outside = false;
            Bx[k] = b;
        }
        __syncthreads();
    } else {
        // chunk by chunk: the source box of chunk k + 1 is copied
        // asynchronously into one staging buffer while chunk k is computed
        // from the other, with one barrier per chunk (once chunk k's copies
        // have landed, everyone is also done with chunk k - 1's buffer).  A
        // warp covers a lanes_x x (32 / lanes_x) block of the chunk (shape
        // and staging pitch chosen per rotation to spread its taps over the
        // shared-memory banks); every thread walks down one canvas column,
        // where moving kRowStep rows adds 2 kRowStep (sq, cq) to the Q32
        // source point.
        const float *__restrict__ src = G.src;
        const int sp = G.src_pitch, P = G.stage_pitch, ax = G.lanes_x;
        const int cpb = kChunk / ax;
        const int c = (int)(warp % cpb) * ax + (int)(lane % ax);
        const int rg = (int)(warp / cpb) * (32 / ax) + (int)(lane / ax);
        const long long xlim = (long long)(2 * W - 1) * HALF, ylim = (long long)(2 * H - 1) * HALF;
        const long long dpx = 2LL * kRowStep * G.sq, dpy = 2LL * kRowStep * G.cq;
        // the chunks' source boxes, once per tile: lane group g (four lanes,
        // one corner each) of warp w makes the box of chunk 8 w + g
        for (int base = 0; base < nch; base += kWarpThreads / 4) {
            const int kc = base + (int)(warp * 8u + (lane >> 2)), kk = min(kc, nch - 1);
            const int q0 = kk * kChunk, cn = min(kChunk, cw - q0);
            const StageBox b = chunk_box(Gm, clampi(cx0 + q0, 0, Wr - 1), clampi(cx0 + q0 + cn - 1, 0, Wr - 1), j0,
                                         j1, W, H, lane);
            if (kc < nch && (lane & 3u) == 0u) Bx[kc] = b;
        }
        __syncthreads();
        // Chunks whose source lies wholly outside the image are background:
        // they are written as zeros on the way and take no staging buffer, so
        // the copies of the next staged chunk always overlap a computed one.
        auto next_staged = [&](int k, StageBox &b) {
            for (; k < nch; ++k) {
                b = Bx[k];
                if (!b.outside) break;
                const int q0 = k * kChunk, cn = min(kChunk, cw - q0);
                if (c < cn)
                    for (int r = rg; r < nrows; r += kRowStep) Cs[r * cwp + q0 + c] = 0.f;
            }
            return k;
        };
        StageBox bx;
        int k = next_staged(0, bx), buf = 0;
        if (k < nch) stage_box(Sbuf, P, src, sp, bx, warp, lane);
        cp_async_commit();
        while (k < nch) {
            cp_async_wait<0>();      // this thread's copies of chunk k have landed
            __syncthreads();         // and everyone's; everyone is done with the other buffer (chunk k - 1)
            StageBox nb;
            const int kn = next_staged(k + 1, nb);
            if (kn < nch) stage_box(Sbuf + (buf ^ 1) * kStageBuf, P, src, sp, nb, warp, lane);
            cp_async_commit();
            const float *Ss = Sbuf + buf * kStageBuf;
            const int q0 = k * kChunk, cn = min(kChunk, cw - q0);
            if (c < cn) {
                const int i = clampi(cx0 + q0 + c, 0, Wr - 1);   // strip position -> canvas column (clamped)
                long long px, py;
                Gm.map(i, j0 + rg, px, py);
                float *Cp = Cs + q0 + c;
                if (bx.interior) {
                    for (int r = rg; r < nrows; r += kRowStep, px += dpx, py += dpy)
                        Cp[r * cwp] = interp_interior(Ss, P, px, py, bx.sx0, bx.sy0);
                } else {
                    for (int r = rg; r < nrows; r += kRowStep, px += dpx, py += dpy) {
                        float acc = 0.f;
                        const int x0 = (int)(px >> 32), y0 = (int)(py >> 32);
                        if (x0 >= 2 && x0 + 3 <= W - 1 && y0 >= 2 && y0 + 3 <= H - 1) {
                            acc = interp_interior(Ss, P, px, py, bx.sx0, bx.sy0);
                        } else if (px >= -HALF && px < xlim && py >= -HALF && py < ylim) {
                            float2 w[6];
                            lanczos3_weights2((uint32_t)px, (uint32_t)py, w);
                            int xs[6];
#pragma unroll
                            for (int m = 0; m < 6; ++m) xs[m] = clampi(x0 + m - 2, 0, W - 1) - bx.sx0;
#pragma unroll
                            for (int n = 0; n < 6; ++n) {
                                const float *row = Ss + (clampi(y0 + n - 2, 0, H - 1) - bx.sy0) * P;
                                float a = 0.f;
#pragma unroll
                                for (int m = 0; m < 6; ++m) a = fmaf(w[m].x, row[xs[m]], a);
                                acc = fmaf(w[n].y, a, acc);
                            }
                        }
                        Cp[r * cwp] = acc;
                    }
                }
            }
            k = kn;
            bx = nb;
            buf ^= 1;
        }
        cp_async_wait<0>();
        __syncthreads();             // zero-filled chunks written after the last staged one
    }

    // 2. for every member view: the Gaussian along canvas x, the tilt
    //    resampling, quantisation and the footprint mask.  Both filters act
    //    along canvas x of one row, so per view column x they are one filter
    //    h_x over the canvas columns x0-2-K .. x0+3+K (computed once per view
    //    by tilt_filter_kernel): v(x, j) = sum_u h_x[u] C(x0 - 2 - K + u, j).
    //    A warp covers 8 view columns x 4 rows and each thread its column's
    //    rows rg, rg + 4, rg + 8, rg + 12 (one filter load serves four rows).
    //    A column whose taps lie in background chunks only is 0 with mask 0
    //    (every canvas point there maps outside the image).  The mask needs
    //    canvas columns x0 and x0 + 1 inside the canvas and their source
    //    points inside the shrunk footprint, tracked in Q32 as in step 1.
    const int rg = (int)(lane >> 3);
    const long long xoff = (long long)(Wr - 1) * HALF;
    const long long mxlo = HALF, mxhi = (long long)(2 * W - 3) * HALF;
    const long long mylo = HALF, myhi = (long long)(2 * H - 3) * HALF;
    const unsigned long long mxr = (unsigned long long)(mxhi - mxlo), myr = (unsigned long long)(myhi - mylo);
    const bool fp_any = mxhi >= mxlo && myhi >= mylo;   // the shrunk footprint is empty below 2 x 2 pixels
    const long long dpx = 2LL * kFiltStep * G.sq, dpy = 2LL * kFiltStep * G.cq;
    for (int m = 0; m < G.n_views; ++m) {
        const DevView &V = views[G.view[m]];
        const int xa = mcols[2 * m], xb = mcols[2 * m + 1];
        const int ncols = xb - xa;
        if (ncols <= 0) continue;
        const int K = V.K, hp = V.hp, nh = 2 * K + 6;
        const int fp = (hp & 7) ? hp : hp + 4;   // = 4 mod 8: a warp's 8 columns on distinct banks
        const bool staged = ncols * fp <= 2 * kStageBuf;
        if (staged) {
            for (int cc = (int)warp; cc < ncols; cc += kWarpThreads / 32)
                for (int g = (int)lane; g < (hp >> 2); g += 32)
                    cp_async16(Sbuf + cc * fp + 4 * g, V.filt + (size_t)(xa + cc) * hp + 4 * g);
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
        }
        for (int cb = 0; cb < ncols; cb += kWarpThreads / 4) {
            const int c = cb + (int)(warp * 8 + (lane & 7u));
            if (c < ncols) {
                const int x = xa + c;
                const long long X = V.tq * (2LL * x - V.Wv + 1) + xoff;
                const int x0 = (int)(X >> 32);
                const int p0 = x0 - 2 - K - cx0;   // strip position of the first tap
                bool bg = true;
                for (int kc = p0 / kChunk; kc <= (p0 + nh - 1) / kChunk; ++kc) bg &= Bx[kc].outside;
                float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
                if (!bg) {
                    const float *Cb = Cs + p0 + rg * cwp;
                    const float *h = staged ? Sbuf + c * fp : V.filt + (size_t)x * hp;
#pragma unroll 4
                    for (int u = 0; u < nh; ++u) {
                        const float hu = staged ? h[u] : __ldg(h + u);
                        acc0 = fmaf(hu, Cb[u], acc0);
                        acc1 = fmaf(hu, Cb[4 * cwp + u], acc1);
                        acc2 = fmaf(hu, Cb[8 * cwp + u], acc2);
                        acc3 = fmaf(hu, Cb[12 * cwp + u], acc3);
                    }
                }
                const float accs[4] = {acc0, acc1, acc2, acc3};
                const bool cols_ok = fp_any && !bg && x0 >= 0 && x0 + 1 <= Wr - 1;
                // the source points relative to the footprint's low corner: each
                // coordinate is inside [lo, hi] iff its offset, as unsigned, is <= hi - lo
                long long pxa, pya, pxb, pyb;
                Gm.map(clampi(x0, 0, Wr - 1), j0 + rg, pxa, pya);
                Gm.map(clampi(x0 + 1, 0, Wr - 1), j0 + rg, pxb, pyb);
                pxa -= mxlo;
                pxb -= mxlo;
                pya -= mylo;
                pyb -= mylo;
#pragma unroll
                for (int q = 0; q < kWarpTH / kFiltStep; ++q, pxa += dpx, pya += dpy, pxb += dpx, pyb += dpy) {
                    const int r = rg + q * kFiltStep;
                    if (r >= nrows) break;
                    const int j = j0 + r;
                    const float v = accs[q];
                    const bool valid = cols_ok && (unsigned long long)pxa <= mxr && (unsigned long long)pya <= myr &&
                                       (unsigned long long)pxb <= mxr && (unsigned long long)pyb <= myr;
                    const size_t o = (size_t)V.out_off + (size_t)j * V.Wv + x;
                    if (out_f32) out_f32[o] = v;
                    const int q8 = __float2int_rn(v);
                    out_u8[o] = (uint8_t)min(255, max(0, q8));
                    out_mask[o] = (uint8_t)valid;
                }
            }
        }
        __syncthreads();             // the filters' buffer is reused by the next member
    }
}

// The Gaussian + tilt filter of every view column (one thread per column;
// blockIdx.y = view): X = t (x - (Wv-1)/2) + (Wr-1)/2 in Q32, Lanczos-3 weights
// w_m of the tilt taps at the canvas columns clamp(x0 - 2 + m), and
// h[u] = sum_m w_m g_|off_m + K - u| with off_m = clamp(x0 - 2 + m) - (x0 - 2),
// so that sum_u h[u] C(x0 - 2 - K + u) = sum_m w_m B(clamp(x0 - 2 + m)) with
// B(i) = sum_k g_|k| C(clamp(i - k)) exactly (the canvas strip holds clamped
// columns).  Entries past 2K + 5 are zero.
__global__ void tilt_filter_kernel(const DevView *__restrict__ views)
{
    const DevView &V = views[blockIdx.y];
    const int Wv = V.Wv, Wr = V.Wr, K = V.K, hp = V.hp;
    const long long xoff = (long long)(Wr - 1) * 2147483648LL;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < Wv; x += gridDim.x * blockDim.x) {
        const long long X = V.tq * (2LL * x - Wv + 1) + xoff;
        const int x0 = (int)(X >> 32);
        float w[6];
        lanczos3_weights((uint32_t)X, w);
        int off[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) off[m] = clampi(x0 - 2 + m, 0, Wr - 1) - (x0 - 2);
        float *h = V.filt + (size_t)x * hp;
        for (int u = 0; u < hp; ++u) {
            float s = 0.f;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int k = abs(off[m] + K - u);
                if (k <= K) s = fmaf(w[m], V.g[k], s);
            }
            h[u] = s;
        }
    }
}

// Grid-stride over the tiles: one CTA per tile, or a persistent grid.
__global__ void __launch_bounds__(kWarpThreads, 4)
warp_band_kernel(int n_tiles, const DevRotGroup *__restrict__ groups, int n_groups, const DevView *__restrict__ views,
                 int seg_w, int cwp, uint8_t *__restrict__ out_u8, uint8_t *__restrict__ out_mask,
                 float *__restrict__ out_f32)
{
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        warp_band_tile(tile, groups, n_groups, views, seg_w, cwp, out_u8, out_mask, out_f32);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side
void warp_strip_widths(const asift_view_desc &v, int tw, int *cw, int *bw)
{
    // tilt taps: floor(X) - 2 .. floor(X) + 3 over tw view columns spaced t
    // apart (+1 for the rounding of tq); the C strip adds K on both sides for
    // the Gaussian.
    const int span = (int)std::ceil(v.t * (tw - 1)) + 2;
    *bw = span + 6;
    *cw = *bw + 2 * v.K;
}

// View columns per tile: the rotation step works in chunks of kChunk canvas
// columns, so a strip just past a multiple of kChunk leaves most lanes of its
// last chunk idle.  Pick tw in [32, kWarpTW] minimising the lane-columns of
// all the view's tiles plus a per-tile overhead (worth half a chunk).
int warp_tile_width(const asift_view_desc &v)
{
    int best = kWarpTW;
    long long best_cost = -1;
    for (int tw = kWarpTW; tw >= 32; --tw) {
        int cw, bw;
        warp_strip_widths(v, tw, &cw, &bw);
        const long long tiles = (v.Wv + tw - 1) / tw;
        const long long cost = tiles * ((long long)((cw + kChunk - 1) / kChunk) * kChunk + kChunk / 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = tw;
        }
    }
    return best;
}

int tilt_filter_pitch(int K) { return (2 * K + 6 + 3) & ~3; }

static int strip_pitch(int cw_max) { return ((cw_max + 3) & ~3) + 1; }

size_t warp_band_smem_bytes(int seg_w, int hk_max)
{
    return sizeof(float) * ((size_t)kWarpTH * strip_pitch(seg_w + 2 * hk_max) + (size_t)2 * kStageBuf) +
           sizeof(StageBox) * kMaxChunks;
}

// Canvas columns per band tile: a segment keeps the strip (seg_w + 2 hK
// columns) and the staging buffers at four CTAs per SM.
int warp_seg_width_default() { return 576; }

bool warp_seg_width_ok(int seg_w, int hk_max)
{
    return seg_w >= kChunk && seg_w <= 1024 && (seg_w + 2 * hk_max + kChunk - 1) / kChunk <= kMaxChunks;
}

// Groups of the views that share a rotated canvas: the same source image and
// the same (cq, sq, Wr, Hr).  per_view: one group per view (each launched on
// its own, tile_start 0).  Members keep the order of the view list.
void build_rot_groups(const asift_view_desc *h, const DevView *dv, int nv, bool per_view, int seg_w,
                      std::vector<DevRotGroup> &out, int *n_tiles, int *hk_max)
{
    out.clear();
    std::map<std::tuple<const float *, long long, long long, int, int>, int> open;
    for (int v = 0; v < nv; ++v) {
        const auto key = std::make_tuple(dv[v].src, h[v].cq, h[v].sq, h[v].Wr, h[v].Hr);
        auto it = per_view ? open.end() : open.find(key);
        if (it == open.end() || out[it->second].n_views == kGroupMax) {
            DevRotGroup g{};
            g.src = dv[v].src;
            g.src_pitch = dv[v].src_pitch;
            g.W = h[v].W;
            g.H = h[v].H;
            g.Wr = h[v].Wr;
            g.Hr = h[v].Hr;
            g.cq = h[v].cq;
            g.sq = h[v].sq;
            g.lanes_x = dv[v].lanes_x;
            g.stage_pitch = dv[v].stage_pitch;
            g.identity = (h[v].cq == (1LL << 31) && h[v].sq == 0) ? 1 : 0;
            out.push_back(g);
            if (!per_view) open[key] = (int)out.size() - 1;
            it = per_view ? open.end() : open.find(key);
        }
        DevRotGroup &g = per_view ? out.back() : out[it->second];
        g.view[g.n_views++] = v;
    }
    int tiles = 0, hk = 3;
    for (DevRotGroup &g : out) {
        int km = 0;
        for (int m = 0; m < g.n_views; ++m) km = std::max(km, h[g.view[m]].K);
        g.hK = km + 3;
        g.nseg = (g.Wr + seg_w - 1) / seg_w;
        g.nbands = (g.Hr + kWarpTH - 1) / kWarpTH;
        g.tile_start = per_view ? 0 : tiles;
        tiles += g.nseg * g.nbands;
        hk = std::max(hk, g.hK);
    }
    *n_tiles = tiles;
    *hk_max = hk;
}

// The rotation step's warp footprint (lanes_x canvas columns x 32 / lanes_x
// rows) and staging pitch for a rotation (cq, sq): the pair whose 32 tap
// base addresses fall on the fewest distinct addresses per shared-memory bank
// (the worst bank decides a load's wavefronts), averaged over 64 sub-pixel
// offsets of the footprint.  Ties go to the smaller pitch, then wider rows.
static void lane_layout_search(long long cq, long long sq, int *lanes_x, int *pitch)
{
    const double c = (double)cq / 2147483648.0, s = (double)sq / 2147483648.0;
    double best = 1e30;
    *lanes_x = 32;
    *pitch = kPitchMin;
    for (int ax : {32, 16, 8}) {
        for (int P = kPitchMin; P <= kPitchMax; P += 4) {
            double tot = 0.0;
            for (int o = 0; o < 64; ++o) {
                const double ox = ((o & 7) + 0.5) / 8.0, oy = ((o >> 3) + 0.5) / 8.0;
                long long addr[32];
                for (int L = 0; L < 32; ++L) {
                    const int di = L % ax, dj = L / ax;
                    const long long x = (long long)std::floor(c * di + s * dj + ox);
                    const long long y = (long long)std::floor(-s * di + c * dj + oy);
                    addr[L] = y * P + x;
                }
                int worst = 0;
                for (int b = 0; b < 32; ++b) {
                    long long seen[32];
                    int n = 0;
                    for (int L = 0; L < 32; ++L) {
                        if ((((addr[L] % 32) + 32) % 32) != b) continue;
                        bool dup = false;
                        for (int q = 0; q < n; ++q) dup |= seen[q] == addr[L];
                        if (!dup) seen[n++] = addr[L];
                    }
                    worst = std::max(worst, n);
                }
                tot += worst;
            }
            if (tot < best - 1e-9) {
                best = tot;
                *lanes_x = ax;
                *pitch = P;
            }
        }
    }
}

// The search is memoised by rotation: view tables repeat the same few dozen
// angles for every image.
void warp_lane_layout(long long cq, long long sq, int *lanes_x, int *pitch)
{
    static std::mutex mu;
    static std::map<std::pair<long long, long long>, std::pair<int, int>> memo;
    const auto key = std::make_pair(cq, sq);
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto it = memo.find(key);
        if (it != memo.end()) {
            *lanes_x = it->second.first;
            *pitch = it->second.second;
            return;
        }
    }
    lane_layout_search(cq, sq, lanes_x, pitch);
    std::lock_guard<std::mutex> lock(mu);
    memo.emplace(key, std::make_pair(*lanes_x, *pitch));
}

cudaError_t launch_u8_to_f32(const uint8_t *src, int pitch, int W, int H, float *dst, int dpitch, cudaStream_t s)
{
    const long long n = (long long)dpitch * H;
    int blocks = (int)std::min<long long>((n + 255) / 256, 8LL * device_sm_count());
    u8_to_f32_kernel<<<blocks, 256, 0, s>>>(src, pitch, W, H, dst, dpitch);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_convert_images(const ImageConv *d_list, int n, long long max_px, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int bx = (int)std::max<long long>(1, std::min<long long>((max_px + 255) / 256, 4LL * device_sm_count()));
    convert_images_kernel<<<dim3(bx, n), 256, 0, s>>>(d_list);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tilt_filter(const DevView *d_views, int n_views, int max_wv, cudaStream_t s)
{
    if (n_views <= 0 || max_wv <= 0) return cudaSuccess;
    tilt_filter_kernel<<<dim3((max_wv + 127) / 128, n_views), 128, 0, s>>>(d_views);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_warp(const DevRotGroup *d_groups, int n_groups, const DevView *d_views, int n_tiles, int seg_w,
                        int hk_max, uint8_t *u8, uint8_t *mask, float *f32, cudaStream_t s, int grid)
{
    if (n_tiles <= 0 || n_groups <= 0) return cudaSuccess;
    if (!warp_seg_width_ok(seg_w, hk_max)) return cudaErrorInvalidValue;
    const size_t smem = warp_band_smem_bytes(seg_w, hk_max);
    const cudaError_t e = ensure_dynamic_smem((const void *)warp_band_kernel, smem);
    if (e != cudaSuccess) return e;
    const int g = (grid > 0 && grid < n_tiles) ? grid : n_tiles;
    warp_band_kernel<<<g, kWarpThreads, smem, s>>>(n_tiles, d_groups, n_groups, d_views, seg_w,
                                                    strip_pitch(seg_w + 2 * hk_max), u8, mask, f32);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asift
