// orb.cu -- ORB on every simulated view (Sec. III-B; ORB [23]) on sm_103a.
//
// Stages, each one launch over all (view, level) entries of a call:
//   mask_rows_kernel    level 0: each row's hull of mask-valid columns
//   hull_levels_kernel  levels >= 1: the hulls implied through the pyramid's
//                       taps (a superset of the valid set), every level at
//                       once from level 0's
//   pyramid_kernel      level l from level l-1: centre-aligned integer bilinear
//                       (Q11 weights, round half up) + AND of the four mask taps
//                       (a view whose masks are its row hulls needs no plane)
//   det_list_kernel     the detection tiles whose rows the hulls leave open
//   detect_kernel       FAST-9 + Harris x25 + 3x3 NMS on shared-memory tiles of
//                       that list; survivors appended with a warp-aggregated
//                       atomic
//   select_kernel       per (view, level): exact top-q by (R25 desc, y, x) via
//                       MSD radix select on a 96-bit key + bitonic sort
//   pool_scan_kernel    canonical pool offsets (view, level, rank)
//   orient_brief_kernel one warp per keypoint: 37x37 patch in shared memory,
//                       integer smoothing, centroid moments -> 30-bin angle,
//                       steered BRIEF-256 packed with warp ballots
// All arithmetic is integer, so the results are exactly those of the
// definitions (and of any independent implementation of them).
#include "common.cuh"
#include "kernels.h"

namespace asift {

// ---------------------------------------------------------------- pyramid
// Each CTA makes a kPyrTW x kPyrTH tile of level l: warp w owns rows
// kPyrRowsW w .. + kPyrRowsW - 1 of it and lane k columns 4k .. 4k + 3, so a
// thread computes its four columns' source taps once and reuses them on every
// row; a row's taps are computed by one lane and broadcast.  Parent pixels
// are read straight from the previous level (just written, so L2-resident);
// each output pixel is eight byte loads and integer FMAs, and four pixels go
// out as one word per plane where the row allows.
constexpr int kPyrRowsW = kPyrTH / 8;

// Centre-aligned source tap of output position o on a level of nl samples
// whose parent has np: ((2o + 1) np - nl) / (2 nl) as q0 + f / 2048 (f the
// Q11 fraction, rounded down), q1 = min(q0 + 1, np - 1).  The integer
// quotients come from a float reciprocal and one correction step, exact
// because the float quotient is within one of the true one.
__device__ __forceinline__ int div_floor(int num, int den, float inv, int &rem)
{
    int q = __float2int_rz((float)num * inv);
    int r = num - q * den;
    if (r < 0) {
        --q;
        r += den;
    } else if (r >= den) {
        ++q;
        r -= den;
    }
    rem = r;
    return q;
}

__device__ __forceinline__ void pyr_tap(int o, int nl, int np, float inv, int &q0, int &q1, int &f)
{
    const int den = 2 * nl;
    int r, r2;
    q0 = div_floor((2 * o + 1) * np - nl, den, inv, r);
    f = div_floor(r << 11, den, inv, r2);
    q1 = min(q0 + 1, np - 1);
}

__device__ __forceinline__ void pyramid_tile(int tile, const DevLevel *__restrict__ lv, int n,
                                             const int32_t *__restrict__ unit)
{
    const int e = find_owner(lv, n, tile, [](const DevLevel &d) { return d.pyr_tile_start; });
    const DevLevel &L = lv[e];
    const int lt = tile - L.pyr_tile_start;
    const int ty = lt / L.pyr_ntx, tx = lt - ty * L.pyr_ntx;
    const int Wl = L.W, Hl = L.H, Wp = L.Wp, Hp = L.Hp;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const int xb = tx * kPyrTW + 4 * (int)lane;
    const int yb = ty * kPyrTH + (int)warp * kPyrRowsW;
    if (yb >= Hl) return;   // warp-uniform; no barrier follows
    const float invx = __frcp_rn((float)(2 * Wl)), invy = __frcp_rn((float)(2 * Hl));
    int x0[4], x1[4], fx[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        pyr_tap(min(xb + c, Wl - 1), Wl, Wp, invx, x0[c], x1[c], fx[c]);
    }
    int ry0 = 0, ry1 = 0, rfy = 0;
    if ((int)lane < kPyrRowsW) pyr_tap(min(yb + (int)lane, Hl - 1), Hl, Hp, invy, ry0, ry1, rfy);
    const int nx = min(4, Wl - xb);   // this lane's columns inside the level (may be <= 0)
    const uint8_t *__restrict__ prev = L.prev;
    const uint8_t *__restrict__ prevm = L.prev_mask;
    const bool planes = __ldg(unit + L.view) == 0;   // unit-convex views keep their masks as row hulls only
    const bool pairs = x1[0] == x0[0] + 1 && x1[1] == x0[1] + 1 && x1[2] == x0[2] + 1 && x1[3] == x0[3] + 1;
#pragma unroll 1
    for (int r = 0; r < kPyrRowsW; ++r) {
        const int y = yb + r;
        const int y0 = __shfl_sync(0xffffffffu, ry0, r), y1 = __shfl_sync(0xffffffffu, ry1, r);
        const unsigned fy = (unsigned)__shfl_sync(0xffffffffu, rfy, r), gy = 2048u - fy;
        if (y >= Hl) break;   // warp-uniform
        if (nx <= 0) continue;
        const uint8_t *P0 = prev + (size_t)y0 * Wp, *P1 = prev + (size_t)y1 * Wp;
        uint32_t wi = 0, wm = 0;
        if (pairs) {   // x1 = x0 + 1 in all four columns: one address per tap pair
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint8_t *q0 = P0 + x0[c], *q1 = P1 + x0[c];
                const unsigned a = __ldg(q0), b = __ldg(q0 + 1), cc = __ldg(q1), d = __ldg(q1 + 1);
                const unsigned f = (unsigned)fx[c], g = 2048u - f;
                const unsigned sum = gy * (g * a + f * b) + fy * (g * cc + f * d);
                wi |= ((sum + (1u << 21)) >> 22) << (8 * c);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const unsigned a = __ldg(P0 + x0[c]), b = __ldg(P0 + x1[c]);
                const unsigned cc = __ldg(P1 + x0[c]), d = __ldg(P1 + x1[c]);
                const unsigned f = (unsigned)fx[c], g = 2048u - f;
                const unsigned sum = gy * (g * a + f * b) + fy * (g * cc + f * d);
                wi |= ((sum + (1u << 21)) >> 22) << (8 * c);
            }
        }
        if (planes) {
            const uint8_t *M0 = prevm + (size_t)y0 * Wp, *M1 = prevm + (size_t)y1 * Wp;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const unsigned m = __ldg(M0 + x0[c]) & __ldg(M0 + x1[c]) & __ldg(M1 + x0[c]) & __ldg(M1 + x1[c]);
                wm |= m << (8 * c);
            }
        }
        uint8_t *oi = L.img_w + (size_t)y * Wl + xb, *om = L.mask_w + (size_t)y * Wl + xb;
        if (nx == 4 && ((((uintptr_t)oi) | ((uintptr_t)om)) & 3u) == 0u) {
            *reinterpret_cast<uint32_t *>(oi) = wi;
            if (planes) *reinterpret_cast<uint32_t *>(om) = wm;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < nx) {
                    oi[c] = (uint8_t)(wi >> (8 * c));
                    if (planes) om[c] = (uint8_t)(wm >> (8 * c));
                }
        }
    }
}

// Grid-stride over the tiles: one CTA per tile, or a persistent grid.
__global__ void __launch_bounds__(256, 4)
pyramid_kernel(int n_tiles, const DevLevel *__restrict__ lv, int n, const int32_t *__restrict__ unit)
{
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) pyramid_tile(tile, lv, n, unit);
}

// ---------------------------------------------------------------- mask row hulls
// Level 0 of every view (the entries 0 .. n - 1): one warp per row finds the
// first and last column whose mask is nonzero (lo > hi when none).  The row's
// 16-byte aligned interior is read as uint4 (independent loads, so that a
// row takes one or two memory latencies), its ragged ends byte by byte.  The
// warp also counts the row's nonzero bytes and its bytes equal to 1: a view
// whose every row has all its nonzero bytes equal to 1 and exactly on
// [lo, hi] (the views' footprints do) is "unit-convex", unit[view] stays
// nonzero, and then every level's mask is 1 exactly on its row hulls (the
// pyramid's AND of four taps keeps rows 0/1 intervals), so the pyramid and the
// detection can work from the hulls instead of the mask planes.
__device__ __forceinline__ void hull_word(uint32_t w, int c, int &lo, int &hi, int &nz, int &n1)
{
    if (w) {
        lo = min(lo, c + ((__ffs((int)w) - 1) >> 3));
        hi = max(hi, c + ((31 - __clz((int)w)) >> 3));
        // bit 7 of each byte: the byte is nonzero / the byte is 1
        nz += __popc((((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u);
        const uint32_t t = w ^ 0x01010101u;
        n1 += __popc(~((((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t)) & 0x80808080u);
    }
}

__global__ void __launch_bounds__(256)
mask_rows_kernel(const DevLevel *__restrict__ lv, int n, int rows, int32_t *__restrict__ row_lo,
                 int32_t *__restrict__ row_hi, int32_t *__restrict__ unit)
{
    const int lane = threadIdx.x & 31;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < rows; g += (gridDim.x * blockDim.x) >> 5) {
        const int e = find_owner(lv, n, g, [](const DevLevel &d) { return d.row_off; });
        const DevLevel &L = lv[e];
        const int W = L.W;
        const uint8_t *__restrict__ m = L.mask + (size_t)(g - L.row_off) * W;
        const int head = min(W, (int)((16 - ((uintptr_t)m & 15u)) & 15u));   // bytes before the first aligned chunk
        const int n16 = (W - head) >> 4;                                     // aligned 16-byte chunks
        const int tail0 = head + 16 * n16;                                   // first byte after them
        int lo = kHullEmptyLo, hi = kHullEmptyHi, nz = 0, n1 = 0;
        if (lane < head) {                                                    // the ragged ends, bytewise
            const int v = __ldg(m + lane);
            if (v) { lo = lane; hi = lane; ++nz; n1 += v == 1; }
        }
        for (int c = tail0 + lane; c < W; c += 32) {
            const int v = __ldg(m + c);
            if (v) { lo = min(lo, c); hi = max(hi, c); ++nz; n1 += v == 1; }
        }
        const uint4 *__restrict__ m16 = reinterpret_cast<const uint4 *>(m + head);
        for (int k = lane; k < n16; k += 32) {
            const uint4 v = __ldg(m16 + k);
            const int c = head + 16 * k;
            hull_word(v.x, c, lo, hi, nz, n1);
            hull_word(v.y, c + 4, lo, hi, nz, n1);
            hull_word(v.z, c + 8, lo, hi, nz, n1);
            hull_word(v.w, c + 12, lo, hi, nz, n1);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            nz += __shfl_xor_sync(0xffffffffu, nz, o);
            n1 += __shfl_xor_sync(0xffffffffu, n1, o);
        }
        if (lane == 0) {
            row_lo[g] = lo;
            row_hi[g] = hi;
            if (nz != n1 || (nz != 0 && nz != hi - lo + 1)) atomicAnd(unit + L.view, 0);
        }
    }
}

// Levels >= 1: a level-l pixel's mask is the AND of the previous level's at
// the pyramid's four taps (columns x0(x), x1(x), rows y0(y), y1(y)), so it can
// be 1 only if x0 >= max(lo(y0), lo(y1)) = A and x1 <= min(hi(y0), hi(y1)) = B;
// x0 and x1 grow with x, so those x form an interval [F(A), G(B)].  With
// x0(x) = floor(((2x + 1) Wp - Wl) / (2 Wl)) (the numerator is >= 0),
// x0(x) >= A  <=>  x >= ceil((2 Wl A + Wl - Wp) / (2 Wp)), and
// x1(x) = min(x0(x) + 1, Wp - 1) > B  <=>  x0(x) >= B when B < Wp - 1 (never
// otherwise).  The interval holds every valid column (exactly them when the
// previous level's rows are intervals, as the views' masks are).
//   F and G do not decrease, so F(max(a, b)) = max(F(a), F(b)) and G(min) =
// min(G): level l's hull of row y is F_l(...F_1(max lo_0)) and G_l(...G_1(min
// hi_0)) over the level-0 rows reached from y through l steps of the row taps,
// a contiguous range (consecutive y0 differ by 1 or 2).  An empty parent row
// (A > B gives F(A) > G(B)) leaves every row built on it empty, whether it is
// stored as kHullEmpty* or as its own empty interval, so one thread per row
// computes every level at once, with no pass per level.
__device__ __forceinline__ int pyr_tap0(int o, int nl, int np) { return ((2 * o + 1) * np - nl) / (2 * nl); }

// min(first x >= 0 with x0(x) >= A, Wl) for A >= 0: Wl when A >= Wp (x0 < Wp).
__device__ __forceinline__ int first_x_at(int A, int Wl, int Wp)
{
    if (A >= Wp) return Wl;
    const long long n = 2LL * Wl * A + Wl - Wp, d = 2LL * Wp;
    return n <= 0 ? 0 : (int)min((n + d - 1) / d, (long long)Wl);
}

// blockIdx.x: level entry nv + k (levels >= 1); a thread per row.
__global__ void __launch_bounds__(256)
hull_levels_kernel(const DevLevel *__restrict__ lv, int nv, int32_t *__restrict__ row_lo, int32_t *__restrict__ row_hi)
{
    const DevLevel &L = lv[nv + blockIdx.x];
    const int y = blockIdx.y * blockDim.x + threadIdx.x;
    if (y >= L.H) return;
    const int v = L.view, l = L.level;
    int ra = y, rb = y;                                  // the rows reached, level by level down to 0
    for (int k = l; k >= 1; --k) {
        const DevLevel &Q = lv[(size_t)k * nv + v];
        ra = pyr_tap0(ra, Q.H, Q.Hp);
        rb = min(pyr_tap0(rb, Q.H, Q.Hp) + 1, Q.Hp - 1);
    }
    const int off0 = lv[v].row_off;
    int A = 0, B = 0x7fffffff;
    for (int r = ra; r <= rb; ++r) {
        A = max(A, __ldg(row_lo + off0 + r));
        B = min(B, __ldg(row_hi + off0 + r));
    }
    for (int k = 1; k <= l; ++k) {
        const DevLevel &Q = lv[(size_t)k * nv + v];
        const int Wl = Q.W, Wp = Q.Wp;
        A = first_x_at(A, Wl, Wp);
        B = B < 0 ? -1 : (B >= Wp - 1 ? Wl - 1 : first_x_at(B, Wl, Wp) - 1);
    }
    row_lo[L.row_off + y] = A <= B ? A : kHullEmptyLo;
    row_hi[L.row_off + y] = A <= B ? B : kHullEmptyHi;
}

// ---------------------------------------------------------------- staging
// A row copy of the bytes [g, g + n) to shared memory at s, where s and g are
// congruent mod 4, moves aligned words: word k starts at byte 4k - (g mod 4)
// of the row (relative to g; a copy has at most (n + 6) / 4 words), and each
// helper takes that offset from its own pointer.  A word inside the range is
// one 32-bit load and store, the partial words at the two ends predicated
// byte loads and stores, so nothing outside [g, g + n) is read and nothing
// outside [s, s + n) written.
__device__ __forceinline__ uint32_t load_word(const uint8_t *__restrict__ g, int n, int k)
{
    const int lo = 4 * k - (int)((uintptr_t)g & 3u);
    if (lo >= 0 && lo + 4 <= n) return __ldg(reinterpret_cast<const uint32_t *>(g + lo));
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (lo + j >= 0 && lo + j < n) v |= (uint32_t)__ldg(g + lo + j) << (8 * j);
    return v;
}

__device__ __forceinline__ void store_word(uint8_t *s, int n, int k, uint32_t v)
{
    const int lo = 4 * k - (int)((uintptr_t)s & 3u);
    if (lo >= 0 && lo + 4 <= n) {
        *reinterpret_cast<uint32_t *>(s + lo) = v;
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (lo + j >= 0 && lo + j < n) s[lo + j] = (uint8_t)(v >> (8 * j));
}

// ---------------------------------------------------------------- detection
constexpr int kHalo = 5;                        // FAST (3) / Harris (4) at the ring pixels + 1
constexpr int kSW = kDetTW + 2 * kHalo;         // staged image
constexpr int kSH = kDetTH + 2 * kHalo;
constexpr int kRW = kDetTW + 2, kRH = kDetTH + 2;   // tile + one-pixel ring
constexpr int kDetCols = 64;                    // threads along x; blockDim = kDetCols * kDetRowsPar
constexpr int kDetRowsPar = 4;
// The staged image has a row pitch P in 80..83 congruent to the level's width
// mod 4 and starts at the address of its first pixel mod 4, so that aligned
// words of a level row land on aligned words of the stage; a row's whole
// containing words (up to 3 bytes either side) fit between the rows.  The
// tile code is instantiated once per pitch so that the stencil offsets stay
// compile-time constants.
constexpr int kSPMin = kSW + 6, kSPMax = kSPMin + 3;

constexpr int kStageBytes = (kSH * kSPMax + 15) & ~15;
struct DetSmem {
    union {                      // the survivors are read before any response is written
        long long R[kRH][kRW];
        int16_t surv[kRH * kRW]; // compass survivors
    };
    int16_t clist[kRH * kRW];
    __align__(16) uint8_t img[kStageBytes];   // the tile's stage
    uint32_t isc[kRH][(kRW + 31) / 32];   // corner flags of the tile + ring, one bit per column
    uint32_t eab[kRH];   // per tile + ring row: columns a .. b whose FAST corners can be mask-valid, a | b << 16
    int ncl, ncand;
};

// The tile's geometry and stage layout, shared by its preparation and its
// processing.
struct DetGeom {
    int x0, y0, W, H, s0;
    bool interior, wide;
    const uint8_t *g0;
};

__device__ __forceinline__ DetGeom det_geom(const DevLevel &L, const DetItem it)
{
    DetGeom G;
    G.W = L.W;
    G.H = L.H;
    G.x0 = it.x0;
    G.y0 = it.y0;
    G.interior = G.x0 - kHalo >= 0 && G.y0 - kHalo >= 0 && G.x0 + kDetTW + kHalo <= G.W && G.y0 + kDetTH + kHalo <= G.H;
    G.wide = G.interior && G.x0 - kHalo >= 3 && G.x0 + kDetTW + kHalo + 3 <= G.W;
    G.g0 = G.interior ? L.img + (size_t)(G.y0 - kHalo) * G.W + (G.x0 - kHalo) : L.img;
    G.s0 = G.interior ? (int)((uintptr_t)G.g0 & 3u) : 0;
    return G;
}

// Columns c of ring row r (y = y0 - 1 + r, x = x0 - 1 + c) where FAST corners
// can be mask-valid: inside the 16 px border, with x - 16 and x + 16 inside
// the row hulls of y - 16 and y + 16 (a > b when none).
__device__ __forceinline__ void det_row_cols(const DevLevel &L, int x0, int y0, int r, const int32_t *__restrict__ row_lo,
                                             const int32_t *__restrict__ row_hi, int &a, int &b)
{
    const int y = y0 - 1 + r, W = L.W, H = L.H;
    a = 1;
    b = 0;
    if (y >= kBorder && y < H - kBorder) {
        const int lo = max(__ldg(row_lo + L.row_off + y - kBorder), __ldg(row_lo + L.row_off + y + kBorder));
        const int hi = min(__ldg(row_hi + L.row_off + y - kBorder), __ldg(row_hi + L.row_off + y + kBorder));
        const int xa = max(kBorder, lo + kBorder), xb = min(W - kBorder - 1, hi - kBorder);
        a = max(xa - (x0 - 1), 0);
        b = min(xb - (x0 - 1), kRW - 1);
    }
}

// 1 iff 9 cyclically consecutive bits of the 16-bit mask m are set.
__device__ __forceinline__ bool has_run9(unsigned m)
{
    m |= m << 16;
    unsigned r = m & (m >> 1);     // 2
    r &= r >> 2;                    // 4
    r &= r >> 4;                    // 8
    r &= m >> 8;                    // 9
    return r != 0u;
}

// FAST-9 at the staged pixel p (row pitch P): the Bresenham circle of radius
// 3 from (0,-3) clockwise, with compile-time offsets.  A 9-arc holds at least
// 2 of the 4 compass points, so pixels with fewer bright and fewer dark
// compass points cannot pass (compass2); fast9_ring is the full test.
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// The compass test of two pixels at once, one per 16-bit lane (values 0..255):
// centres c, compass points n, e, s, w.  At least two of the four points are
// brighter than c + thr iff the second largest is, and at least two darker
// than c - thr iff the second smallest is; of four values, with A the smaller
// of the two pair maxima and B the larger of the two pair minima, the second
// largest is max(A, B) and the second smallest min(A, B).  With kp = 511 - thr
// in each lane (0 <= thr <= 255), hi + kp - c and c + kp - lo lie in [1, 766]
// in every lane, so the 32-bit sums carry and borrow nothing between the
// lanes, and reach 512 (bit 9 of the lane) exactly when hi > c + thr, resp.
// lo < c - thr.  Returns bits 9 and 25: the pixels passing.
__device__ __forceinline__ uint32_t compass2(uint32_t c, uint32_t n, uint32_t e, uint32_t s, uint32_t w, uint32_t kp)
{
    const uint32_t A = vmin2(vmax2(n, e), vmax2(s, w)), B = vmax2(vmin2(n, e), vmin2(s, w));
    const uint32_t hi = vmax2(A, B), lo = vmin2(A, B);
    return ((hi + kp - c) | (c + kp - lo)) & 0x02000200u;
}

// The full FAST-9 test at a compass survivor: ring point k of the circle in
// lane 0 and point k + 8 in lane 1 of a 16-bit pair, both tests per pair
// with the compass test's offset kp (bit 9 of each lane), gathered into the
// 16-bit masks of brighter and darker points.
template <int P>
__device__ __forceinline__ bool fast9_ring(const uint8_t *p, uint32_t kp)
{
    const uint32_t c2 = (uint32_t)p[0] * 0x00010001u;
    const uint32_t v[16] = {p[-3 * P], p[-3 * P + 1], p[-2 * P + 2], p[-P + 3], p[3], p[P + 3], p[2 * P + 2],
                            p[3 * P + 1], p[3 * P], p[3 * P - 1], p[2 * P - 2], p[P - 3], p[-3], p[-P - 3],
                            p[-2 * P - 2], p[-3 * P - 1]};
    uint32_t yb = 0u, yd = 0u;   // bits k and 16 + k: points k and k + 8
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t pr = v[k] | v[k + 8] << 16;
        yb |= ((pr + kp - c2) >> (9 - k)) & (0x00010001u << k);
        yd |= ((c2 + kp - pr) >> (9 - k)) & (0x00010001u << k);
    }
    return has_run9(__byte_perm(yb, 0u, 0x4420)) || has_run9(__byte_perm(yd, 0u, 0x4420));
}

// Preparation of a listed tile: its columns per ring row, and its stage:
// staged pixel (r, c) = image (x0 - kHalo + c, y0 - kHalo + r), clamped, at
// S[r * P + c].  Interior tiles with 3 spare columns of the level on either
// side copy each row's whole containing words asynchronously (every word
// inside the level row; one commit group); other interior tiles copy words
// with byte-exact edges; the rest copy bytes with clamping.
__device__ __forceinline__ void det_prepare(const DetItem it, const DetGeom &G, const DevLevel *__restrict__ lv,
                                            const int32_t *__restrict__ row_lo, const int32_t *__restrict__ row_hi,
                                            DetSmem &sm)
{
    constexpr int kThreads = kDetCols * kDetRowsPar;
    const DevLevel &L = lv[it.e];
    const int P = kSPMin + (G.W & 3);
    if (threadIdx.x < kRH) {
        int a, b;
        det_row_cols(L, G.x0, G.y0, (int)threadIdx.x, row_lo, row_hi, a, b);
        sm.eab[threadIdx.x] = a <= b ? (uint32_t)a | (uint32_t)b << 16 : 1u;   // none: a = 1 > b = 0
    }
    uint8_t *S = sm.img + G.s0;
    if (G.wide) {
        constexpr int kNW = (kSW + 6) / 4;   // words of a row copy
        for (int el = threadIdx.x; el < kSH * kNW; el += kThreads) {
            const int r = el / kNW, k = el - r * kNW;
            const uint8_t *g = G.g0 + (size_t)r * G.W;
            const int mis = (int)((uintptr_t)g & 3u);
            if (4 * k < mis + kSW)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                                 (uint32_t)__cvta_generic_to_shared(S + r * P - mis + 4 * k)),
                             "l"(g - mis + 4 * k)
                             : "memory");
        }
    } else if (G.interior) {
        constexpr int kNW = (kSW + 6) / 4;   // words of a row copy
        for (int el = threadIdx.x; el < kSH * kNW; el += kThreads) {
            const int r = el / kNW, k = el - r * kNW;
            store_word(S + r * P, kSW, k, load_word(G.g0 + (size_t)r * G.W, kSW, k));
        }
    } else {
        const uint8_t *__restrict__ I = L.img;
        const int W = G.W, H = G.H;
        for (int el = threadIdx.x; el < kSH * kSW; el += kThreads) {
            const int r = el / kSW, c = el - r * kSW;
            S[r * P + c] = I[clampi(G.y0 - kHalo + r, 0, H - 1) * W + clampi(G.x0 - kHalo + c, 0, W - 1)];
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// A prepared tile (its stage and row columns visible, counters zeroed):
// FAST, Harris, NMS and the candidates.
template <int P>
__device__ __forceinline__ void det_process(const DetItem it, const DetGeom &G, const DevLevel *__restrict__ lv, int thr,
                                            Candidate *__restrict__ cand, int32_t *__restrict__ cand_count,
                                            const int32_t *__restrict__ unit, DetSmem &sm)
{
    auto &isc = sm.isc;
    auto &R = sm.R;
    int16_t *clist = sm.clist;
    int &ncl = sm.ncl;
    const int e = it.e;
    const DevLevel &L = lv[e];
    const int x0 = G.x0, y0 = G.y0, W = G.W;
    const uint32_t *eab = sm.eab;
    const uint8_t *S = sm.img + G.s0;
    constexpr int kThreads = kDetCols * kDetRowsPar;

    // corner flags on the tile + ring in two passes, so that the full ring test
    // runs with every lane busy: (a) border and compass test for every pixel,
    // survivors listed; (b) the full test and the mask corners on the list,
    // appended with one shared atomic per warp (every lane runs every
    // iteration).
    const unsigned lane_id = threadIdx.x & 31u;
    // (a) four pixels of a ring row per thread and pass: the aligned stage
    // word holding them, its two neighbours in the row and the words three
    // rows up and down give the pixels and their compass points as 16-bit
    // lane pairs (even and odd pixels).  Bit 4k + i of the thread's mask is
    // pixel i of its group in pass k; the survivors are appended once at the
    // end with a warp scan and one atomic per warp.
    int16_t *surv = sm.surv;
    constexpr int kGW = (kRW + 6) / 4;   // groups per ring row: the row's columns after up to 3 of lead-in
    constexpr int kGPass = (kRH * kGW + kThreads - 1) / kThreads;
    static_assert(4 * kGPass <= 32, "a thread's compass results fit one word");
    constexpr int kNm = (4 - (3 * P) % 4) % 4;   // offset of the window three rows up in its aligned word
    constexpr int kSm = (3 * P) % 4;             // and of the window three rows down
    const uint8_t *img = sm.img;                 // ring pixel (r, c) at byte s0 + (r + 4) P + c + 4
    auto word = [&](int off) { return *reinterpret_cast<const uint32_t *>(img + off); };
    const uint32_t kp = (uint32_t)(511 - thr) * 0x00010001u;
    unsigned bits = 0u;
#pragma unroll 1
    for (int k = 0; k < kGPass; ++k) {
        const int el = (int)threadIdx.x + k * kThreads;
        const int r = el / kGW, g = el - r * kGW;
        if (r >= kRH) break;
        const uint32_t ab = eab[r];
        const int q = G.s0 + (r + 4) * P + 4;    // ring column 0
        const int cb = 4 * g - (q & 3);          // ring column of the group's pixel 0
        const int lo = (int)(ab & 0xffffu) - cb, hi = (int)(ab >> 16) - cb;
        const uint32_t m = (0xFu << min(max(lo, 0), 4)) & (0xFu >> min(max(3 - hi, 0), 4));
        if (m == 0u) continue;
        const int wa = (q & ~3) + 4 * g;
        const uint32_t w1 = word(wa);
        const uint32_t ww = __funnelshift_r(word(wa - 4), w1, 8), we = __funnelshift_r(w1, word(wa + 4), 24);
        const uint32_t wn = kNm ? __funnelshift_r(word(wa - 3 * P - kNm), word(wa - 3 * P - kNm + 4), 8 * kNm)
                                : word(wa - 3 * P);
        const uint32_t ws = kSm ? __funnelshift_r(word(wa + 3 * P - kSm), word(wa + 3 * P - kSm + 4), 8 * kSm)
                                : word(wa + 3 * P);
        constexpr uint32_t kEven = 0x00ff00ffu;
        const uint32_t pe = compass2(w1 & kEven, wn & kEven, we & kEven, ws & kEven, ww & kEven, kp);
        const uint32_t po = compass2(__byte_perm(w1, 0u, 0x4341), __byte_perm(wn, 0u, 0x4341), __byte_perm(we, 0u, 0x4341),
                                     __byte_perm(ws, 0u, 0x4341), __byte_perm(ww, 0u, 0x4341), kp);
        const uint32_t t = pe | (po << 1);       // bits 9, 10, 25, 26: pixels 0, 1, 2, 3
        bits |= (((t >> 9) | (t >> 23)) & m) << (4 * k);
    }
    {
        const int cnt = __popc(bits);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane_id >= o) incl += v;
        }
        int base = 0;
        if (lane_id == 31u && incl > 0) base = atomicAdd(&sm.ncand, incl);
        base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
        while (bits) {
            const int b = __ffs((int)bits) - 1;
            bits &= bits - 1u;
            const int el = (int)threadIdx.x + (b >> 2) * kThreads;
            const int r = el / kGW, g = el - r * kGW;
            const int q = G.s0 + (r + 4) * P + 4;
            surv[base++] = (int16_t)(r * kRW + 4 * g + (b & 3) - (q & 3));
        }
    }
    __syncthreads();
    const int nca = sm.ncand;
    const bool unit_view = __ldg(unit + L.view) != 0;
#pragma unroll 1
    for (int q0 = (int)(threadIdx.x & ~31u); q0 < nca; q0 += kThreads) {
        const int q = q0 + (int)lane_id;
        uint8_t flag = 0;
        int r = 0, c = 0;
        if (q < nca) {
            const int el = surv[q];
            r = el / kRW;
            c = el - r * kRW;
            if (fast9_ring<P>(&S[(r - 1 + kHalo) * P + c - 1 + kHalo], kp)) {
                if (unit_view) {
                    flag = 1;   // the row hulls are the mask: eligible = the box's corners mask-valid
                } else {
                    const int x = x0 - 1 + c, y = y0 - 1 + r;
                    const uint8_t *M = L.mask;
                    const int b = kBorder;
                    flag = M[(y - b) * W + x - b] & M[(y - b) * W + x + b] & M[(y + b) * W + x - b] &
                           M[(y + b) * W + x + b];
                }
            }
            if (flag) atomicOr(&isc[r][c >> 5], 1u << (c & 31));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, flag != 0);
        if (bal) {
            int base = 0;
            if (lane_id == 0) base = atomicAdd(&ncl, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (flag) clist[base + __popc(bal & ((1u << lane_id) - 1u))] = (int16_t)(r * kRW + c);
        }
    }
    __syncthreads();
    const int nc = ncl;
    if (nc == 0) return;

    // Harris x25 at every corner of the tile + ring, straight from the staged
    // image, eight lanes per corner: the 7x7 window of Sobel gradients of ring
    // pixel (r, c) (staged (r + 4, c + 4)) reads the 9 x 9 staged pixels from
    // (r, c), and lane s < 7 takes window row s from pixel rows s .. s + 2,
    // with gx = v(x + 1) - v(x - 1) on the column sums v = p0 + 2 p1 + p2 and
    // gy = d(x - 1) + 2 d(x) + d(x + 1) on the row differences d = p2 - p0;
    // the group's sums are exact integers in any order.
    {
        const int sub = (int)(lane_id & 7u), slot = (int)(threadIdx.x >> 3);
#pragma unroll 1
        for (int q0 = 0; q0 < nc; q0 += kThreads / 8) {
            const int q = q0 + slot;
            int a = 0, bb = 0, cc = 0, p = 0;
            if (q < nc) {
                p = clist[q];
                if (sub < 7) {
                    const int r = p / kRW, c = p - r * kRW;
                    const uint8_t *w = S + (r + sub) * P + c;
                    int v[9], d[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int p0 = w[k], p1 = w[P + k], p2 = w[2 * P + k];
                        v[k] = p0 + 2 * p1 + p2;
                        d[k] = p2 - p0;
                    }
#pragma unroll
                    for (int dx = 0; dx < 7; ++dx) {
                        const int ix = v[dx + 2] - v[dx], iy = d[dx] + 2 * d[dx + 1] + d[dx + 2];
                        a += ix * ix;
                        bb += iy * iy;
                        cc += ix * iy;
                    }
                }
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                bb += __shfl_xor_sync(0xffffffffu, bb, o);
                cc += __shfl_xor_sync(0xffffffffu, cc, o);
            }
            if (q < nc && sub == 0) {
                const int r = p / kRW, c = p - r * kRW;
                const long long A = a, B = bb, Cc = cc;
                R[r][c] = 25 * (A * B - Cc * Cc) - (A + B) * (A + B);
            }
        }
    }
    __syncthreads();

    // 3x3 NMS at the corners of the tile proper (the list also holds the
    // ring's); survivors appended with one atomic per warp
    const unsigned lane = threadIdx.x & 31u;
    auto is_corner = [&](int r, int c) { return (isc[r][c >> 5] >> (c & 31)) & 1u; };
#pragma unroll 1
    for (int q0 = (int)(threadIdx.x & ~31u); q0 < nc; q0 += kThreads) {
        const int q = q0 + (int)lane;
        bool keep = false;
        long long rv = 0;
        int x = 0, y = 0;
        if (q < nc) {
            const int p = clist[q];
            const int r = p / kRW, c = p - r * kRW;
            if (r >= 1 && r <= kDetTH && c >= 1 && c <= kDetTW) {
                x = x0 - 1 + c;
                y = y0 - 1 + r;
                rv = R[r][c];
                keep = true;
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        if ((dx | dy) == 0 || !is_corner(r + dy, c + dx)) continue;
                        const long long rn = R[r + dy][c + dx];
                        // the neighbour precedes p in raster order iff dy < 0 or (dy == 0 and dx < 0)
                        const bool n_first = dy < 0 || (dy == 0 && dx < 0);
                        if (!(rv > rn || (rv == rn && !n_first))) keep = false;
                    }
            }
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, keep);
        if (ballot) {
            const int leader = __ffs(ballot) - 1;
            int base = 0;
            if ((int)lane == leader) base = atomicAdd(&cand_count[e], __popc(ballot));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (keep) {
                const int slot = base + __popc(ballot & ((1u << lane) - 1u));
                if (slot < L.cand_cap) {
                    Candidate cd;
                    cd.r25 = rv;
                    cd.yx = (y << 16) | x;
                    cd.pad = 0;
                    cand[L.cand_off + slot] = cd;
                }
            }
        }
    }
}

// The tiles worth detecting on: one block per level entry, a thread per
// tile.  A tile is listed when one of its ring rows has columns where FAST
// corners can be mask-valid (det_row_cols); the others hold no candidate.
__global__ void __launch_bounds__(256)
det_list_kernel(const DevLevel *__restrict__ lv, const int32_t *__restrict__ row_lo, const int32_t *__restrict__ row_hi,
                DetItem *__restrict__ list, int32_t *__restrict__ count)
{
    const int e = blockIdx.x;
    const DevLevel &L = lv[e];
    const int nt = L.det_ntx * ((L.H + kDetTH - 1) / kDetTH);
    const unsigned lane = threadIdx.x & 31u;
    for (int b0 = 0; b0 < nt; b0 += blockDim.x) {
        const int lt = b0 + (int)threadIdx.x;
        bool any = false;
        int x0 = 0, y0 = 0;
        if (lt < nt) {
            const int ty = lt / L.det_ntx, tx = lt - ty * L.det_ntx;
            x0 = tx * kDetTW;
            y0 = ty * kDetTH;
            for (int r = 0; r < kRH && !any; ++r) {
                int a, b;
                det_row_cols(L, x0, y0, r, row_lo, row_hi, a, b);
                any = a <= b;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, any);
        if (bal) {
            int base = 0;
            if (lane == 0) base = atomicAdd(count, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (any) list[base + __popc(bal & ((1u << lane) - 1u))] = DetItem{e, (uint16_t)x0, (uint16_t)y0};
        }
    }
}

// One CTA per listed tile (a positive grid makes it persistent over the list;
// the launch is sized to every tile of the call, and the CTAs past the list's
// count leave at once).  Eight CTAs per SM, what 32 registers and the 26 KB
// of shared memory (the survivors share the responses' space) allow.
// Staging the next tile while processing one, in a persistent grid, was
// slower: tiles differ widely in work, and a fixed stride or a claimed
// counter balances them worse than the hardware's block scheduler.
__global__ void __launch_bounds__(kDetCols * kDetRowsPar, 8)
detect_kernel(const DevLevel *__restrict__ lv, const DetItem *__restrict__ list, const int32_t *__restrict__ count,
              int thr, Candidate *__restrict__ cand, int32_t *__restrict__ cand_count,
              const int32_t *__restrict__ row_lo, const int32_t *__restrict__ row_hi, const int32_t *__restrict__ unit)
{
    __shared__ DetSmem sm;
    const int n = __ldg(count);
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const DetItem cur = list[k];
        const DetGeom G = det_geom(lv[cur.e], cur);
        det_prepare(cur, G, lv, row_lo, row_hi, sm);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (threadIdx.x == 0) {
            sm.ncl = 0;
            sm.ncand = 0;
        }
        if (threadIdx.x < kRH * ((kRW + 31) / 32)) (&sm.isc[0][0])[threadIdx.x] = 0u;
        __syncthreads();
        switch (G.W & 3) {
        case 0: det_process<kSPMin>(cur, G, lv, thr, cand, cand_count, unit, sm); break;
        case 1: det_process<kSPMin + 1>(cur, G, lv, thr, cand, cand_count, unit, sm); break;
        case 2: det_process<kSPMin + 2>(cur, G, lv, thr, cand, cand_count, unit, sm); break;
        default: det_process<kSPMin + 3>(cur, G, lv, thr, cand, cand_count, unit, sm); break;
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------- selection
// Selection key: ascending order = (R25 descending, y ascending, x ascending).
__device__ __forceinline__ unsigned long long key_hi(long long r)
{
    return ~((unsigned long long)r ^ 0x8000000000000000ULL);
}

constexpr int kSelThreads = 512;
constexpr int kSelMax = 4096;   // quota per level <= kSelMax

__global__ void __launch_bounds__(kSelThreads)
select_kernel(const DevLevel *__restrict__ lv, const Candidate *__restrict__ cand,
              const int32_t *__restrict__ cand_count, int n_features, SlotKp *__restrict__ slots,
              int32_t *__restrict__ taken, int32_t *__restrict__ status)
{
    extern __shared__ unsigned char sm_raw[];
    unsigned long long *kh = (unsigned long long *)sm_raw;          // [kSelMax]
    unsigned *kl = (unsigned *)(kh + kSelMax);                      // [kSelMax]
    __shared__ unsigned hist[256];
    __shared__ unsigned long long pre_hi, msk_hi;
    __shared__ unsigned pre_lo, msk_lo;
    __shared__ int need, done, nsel;
    __shared__ int wsum[8];

    const int e = blockIdx.x;
    const DevLevel &L = lv[e];
    int n = cand_count[e];
    if (n > L.cand_cap) {
        if (threadIdx.x == 0) set_status(status, ASIFT_ERR_CAPACITY);
        n = L.cand_cap;
    }
    const int q = L.quota;
    const int k = min(q, n);
    if (threadIdx.x == 0) taken[e] = k;
    if (k == 0) return;
    const Candidate *C = cand + L.cand_off;

    if (threadIdx.x == 0) {
        pre_hi = 0; msk_hi = 0; pre_lo = 0; msk_lo = 0;
        need = k; done = (n <= q); nsel = 0;
    }
    __syncthreads();
    // MSD radix select of the k smallest 96-bit keys (8-bit digits)
    for (int d = 0; d < 12 && !done; ++d) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const unsigned long long ph = pre_hi, mh = msk_hi;
        const unsigned pl = pre_lo, ml = msk_lo;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long h = key_hi(C[i].r25);
            const unsigned l = (unsigned)C[i].yx;
            if ((h & mh) == ph && (l & ml) == pl) {
                const unsigned dig = d < 8 ? (unsigned)(h >> (56 - 8 * d)) & 255u : (l >> (24 - 8 * (d - 8))) & 255u;
                atomicAdd(&hist[dig], 1u);
            }
        }
        __syncthreads();
        // the digit: the first bin b whose inclusive count reaches `need`,
        // from a block scan of the 256 bins (thread b holds bin b)
        {
            const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
            const int v = threadIdx.x < 256 ? (int)hist[threadIdx.x] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += t;
            }
            if (lane == 31u && wid < 8u) wsum[wid] = incl;
            const int nd = need;   // read before the barrier: the winner below rewrites it
            __syncthreads();
            if (threadIdx.x < 256) {
                for (unsigned w = 0; w < wid; ++w) incl += wsum[w];
                const int excl = incl - v;
                if (excl < nd && incl >= nd) {   // exactly one bin
                    const unsigned b = threadIdx.x;
                    need = nd - excl;
                    if (d < 8) {
                        pre_hi |= (unsigned long long)b << (56 - 8 * d);
                        msk_hi |= 255ULL << (56 - 8 * d);
                    } else {
                        pre_lo |= b << (24 - 8 * (d - 8));
                        msk_lo |= 255u << (24 - 8 * (d - 8));
                    }
                    if (v == nd - excl) done = 1;   // the whole bucket is selected
                }
            }
        }
        __syncthreads();
    }
    // threshold: every key <= (prefix with the undecided digits all ones)
    const unsigned long long th = done ? (pre_hi | ~msk_hi) : pre_hi;
    const unsigned tl = done ? (pre_lo | ~msk_lo) : pre_lo;
    const bool all = (n <= q);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long h = key_hi(C[i].r25);
        const unsigned l = (unsigned)C[i].yx;
        if (all || h < th || (h == th && l <= tl)) {
            const int s = atomicAdd(&nsel, 1);
            if (s < kSelMax) { kh[s] = h; kl[s] = l; }
        }
    }
    __syncthreads();
    const int m = min(nsel, kSelMax);
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = m + threadIdx.x; i < P; i += blockDim.x) { kh[i] = ~0ULL; kl[i] = ~0u; }
    __syncthreads();
    // bitonic sort ascending by (hi, lo)
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const bool gt = kh[lo] > kh[hi] || (kh[lo] == kh[hi] && kl[lo] > kl[hi]);
                if (gt == up) {
                    const unsigned long long th2 = kh[lo]; kh[lo] = kh[hi]; kh[hi] = th2;
                    const unsigned tl2 = kl[lo]; kl[lo] = kl[hi]; kl[hi] = tl2;
                }
            }
            __syncthreads();
        }
    }
    SlotKp *out = slots + (size_t)L.view * n_features + L.qoff;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        SlotKp s;
        s.r25 = (long long)(~kh[i] ^ 0x8000000000000000ULL);
        s.yx = (int32_t)kl[i];
        s.e = e;
        out[i] = s;
    }
}

// ---------------------------------------------------------------- pool offsets
// Canonical pool order: view-major, then level, then selection rank.  Views are
// grouped (one group per image); group g owns views [first[g], first[g+1]) and
// the pool slice starting at first[g] * n_features.  One CTA per group.
// Entries of the level table are level-major (index l * n_views + v).
__global__ void __launch_bounds__(1024)
pool_scan_kernel(const int32_t *__restrict__ taken, int n_views, int n_levels, const int32_t *__restrict__ first,
                 int n_features, int32_t *__restrict__ pool_off, int32_t *__restrict__ view_count,
                 int32_t *__restrict__ view_off, int32_t *__restrict__ group_total)
{
    __shared__ int32_t warp_sums[32];
    __shared__ int32_t carry;
    const int g = blockIdx.x;
    const int v0 = first[g], v1 = first[g + 1];
    const int base0 = v0 * n_features;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int n = (v1 - v0) * n_levels;
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;           // canonical index (v - v0) * L + l
        int v = 0, l = 0, val = 0;
        if (i < n) {
            v = v0 + i / n_levels;
            l = i % n_levels;
            val = taken[l * n_views + v];
        }
        int x = val;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int s = (lane < (blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if ((int)lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int excl = carry + x - val + (wid ? warp_sums[wid - 1] : 0);
        if (i < n) {
            pool_off[l * n_views + v] = base0 + excl;
            if (l == 0) view_off[v] = base0 + excl;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + val;
        __syncthreads();
    }
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        int c = 0;
        for (int l = 0; l < n_levels; ++l) c += taken[l * n_views + v];
        view_count[v] = c;
    }
    if (threadIdx.x == 0) group_total[g] = carry;
}

// ---------------------------------------------------------------- orientation + BRIEF
constexpr int kObWarps = 8;
constexpr int kPatch = 37;          // raw patch: radius 15 + smoothing radius 3
constexpr int kPP = 40;             // its row pitch in shared memory (10 words)
constexpr int kSm = 31;             // smoothed patch
// the smoothing taps [18 34 49 54 49 34 18] packed for dp4a: taps 0-3, taps 4-6 (and 0)
constexpr unsigned kTapsLo = 18u | 34u << 8 | 49u << 16 | 54u << 24, kTapsHi = 49u | 34u << 8 | 18u << 16;

// the same taps as byte pairs for dp2a over two 16-bit intermediate values:
// (c0, c1), (c2, c3), (c4, c5), and shifted by one row (0, c0), (c1, c2), (c3, c4), (c5, c6)
constexpr unsigned kV01 = 18u | 34u << 8, kV23 = 49u | 54u << 8, kV45 = 49u | 34u << 8, kV6 = 18u;
constexpr unsigned kW0 = 0u | 18u << 8, kW12 = 34u | 49u << 8, kW34 = 54u | 49u << 8, kW56 = 34u | 18u << 8;
constexpr int kHP = kPatch + 1;     // column pitch of the transposed intermediate (u16; even)

// the disc's half height at column offset |dx| <= 15: the largest hh with
// hh^2 + dx^2 <= 15^2, four bits per |dx|
constexpr int disc_half(int dx)
{
    int hh = 15;
    while (hh * hh > kPatchR2 - dx * dx) --hh;
    return hh;
}
constexpr unsigned long long disc_table()
{
    unsigned long long t = 0;
    for (int d = 0; d <= 15; ++d) t |= (unsigned long long)disc_half(d) << (4 * d);
    return t;
}
constexpr unsigned long long kDiscHalf = disc_table();
static_assert(disc_half(0) == 15 && disc_half(9) == 12 && disc_half(15) == 0, "disc half heights");

__global__ void __launch_bounds__(kObWarps * 32, 7)
orient_brief_kernel(const DevLevel *__restrict__ lv, int n_views, int n_levels, int n_features, int v_begin, int v_end,
                    const SlotKp *__restrict__ slots, const int32_t *__restrict__ taken,
                    const int32_t *__restrict__ pool_off, const int *__restrict__ pattern /* [30][256] packed int8x4 */,
                    const long long *__restrict__ bins /* [30][2] Q30 */, asift_keypoint *__restrict__ kp_out,
                    uint4 *__restrict__ desc_out)
{
    // the smoothed patch S takes the raw patch's place once the horizontal
    // pass and the moments are done with it
    __shared__ __align__(16) uint8_t P[kObWarps][kPatch * kPP];
    __shared__ __align__(16) uint16_t Hs[kObWarps][kSm * kHP];   // horizontal sums, column-major (column c, row r at c kHP + r)
    static_assert(kSm * kSm <= kPatch * kPP, "the smoothed patch fits the raw patch's space");
    __shared__ long long eb[kBins][2];
    for (int i = threadIdx.x; i < kBins * 2; i += blockDim.x) eb[i >> 1][i & 1] = bins[i];
    __syncthreads();

    const int w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const long long slot = (long long)v_begin * n_features + (long long)blockIdx.x * kObWarps + w;
    if (slot >= (long long)v_end * n_features) return;
    const int v = (int)(slot / n_features), rnk = (int)(slot - (long long)v * n_features);
    const SlotKp s = slots[slot];
    // the level whose slot range holds rnk: lane l checks level l (one round
    // of loads instead of a dependent chain over the levels); ranges are disjoint
    bool hit = false;
    if ((int)lane < n_levels) {
        const int ei = (int)lane * n_views + v;
        const int q = lv[ei].qoff;
        hit = rnk >= q && rnk < q + taken[ei];
    }
    const unsigned lv_hit = __ballot_sync(0xffffffffu, hit);
    if (lv_hit == 0u) return;
    const int e = (__ffs((int)lv_hit) - 1) * n_views + v;
    const DevLevel &L = lv[e];
    const int r = rnk - L.qoff;
    const int x = s.yx & 0xffff, y = s.yx >> 16;
    const int W = L.W, H = L.H;

    // patch (rr, cc) = image (x - 18 + cc, y - 18 + rr), clamped, at p[rr * kPP + cc]
    uint8_t *p = P[w];
    if (x >= 22 && x + 26 < W && y >= 18 && y + 18 < H) {
        // rows as words: lane 10 q + j writes word j of rows q, q + 3, ..., each
        // from the two aligned words of the image row around it (both inside
        // the row for keypoints at least 22 px from its ends)
        const int q = (int)lane / 10, j = (int)lane - 10 * q;
#pragma unroll 4   // four rows' loads in flight
        for (int rr = q; rr < kPatch; rr += 3) {
            if (lane >= 30) break;
            const uint8_t *g = L.img + (size_t)(y - 18 + rr) * W + (x - 18);
            const uint32_t *ga = reinterpret_cast<const uint32_t *>(reinterpret_cast<uintptr_t>(g) & ~(uintptr_t)3);
            const unsigned sh = 8u * (unsigned)(reinterpret_cast<uintptr_t>(g) & 3u);
            reinterpret_cast<uint32_t *>(p + rr * kPP)[j] = __funnelshift_r(__ldg(ga + j), __ldg(ga + j + 1), sh);
        }
    } else {
        for (int i = lane; i < kPatch * kPatch; i += 32) {
            const int rr = i / kPatch, cc = i - rr * kPatch;
            const int gx = clampi(x - 18 + cc, 0, W - 1), gy = clampi(y - 18 + rr, 0, H - 1);
            p[rr * kPP + cc] = L.img[(size_t)gy * W + gx];
        }
    }
    __syncwarp();
    // horizontal smoothing pass (exact sums): lane item = (row, 4 consecutive
    // outputs), taps from three aligned words through byte permutes and dp4a
    uint16_t *h = Hs[w];
    for (int i = lane; i < kPatch * 8; i += 32) {
        const int rr = i >> 3, c4 = (i & 7) * 4;
        const uint32_t *row = reinterpret_cast<const uint32_t *>(p + rr * kPP) + (c4 >> 2);
        const uint32_t w0 = row[0], w1 = row[1], w2 = row[2];   // bytes c4 .. c4 + 11 (< kPP)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned sel = 0x3210u + 0x1111u * (unsigned)k;
            const unsigned a = __dp4a(__byte_perm(w1, w2, sel), kTapsHi, __dp4a(__byte_perm(w0, w1, sel), kTapsLo, 0u));
            if (c4 + k < kSm) h[(c4 + k) * kHP + rr] = (uint16_t)a;
        }
    }
    // centroid moments on the raw patch (disc of radius 15): lane dx + 15
    // sums its column over the disc's rows |dy| <= hh (exact integer sums)
    int m10 = 0, m01 = 0;
    if ((int)lane < kSm) {
        const int dx = (int)lane - 15;
        const int hh = (int)((kDiscHalf >> (4 * abs(dx))) & 15ull);
        const uint8_t *col = p + 18 * kPP + dx + 18;   // dy = 0
        int sv = 0, sy = 0;
        for (int dy = -hh; dy <= hh; ++dy) {
            const int val = col[dy * kPP];
            sv += val;
            sy += dy * val;
        }
        m10 = dx * sv;
        m01 = sy;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m10 += __shfl_xor_sync(0xffffffffu, m10, o);
        m01 += __shfl_xor_sync(0xffffffffu, m01, o);
    }
    __syncwarp();
    // vertical pass, rounded half up: lane item = (column, 4 consecutive
    // rows r0 .. r0 + 3), its 10 intermediate values as 5 row pairs of the
    // column-major buffer; each output is dp2a's over the pairs with the taps
    // as byte pairs (exact integer sums; the pad row 37 only reaches row 31,
    // which is not kept)
    uint8_t *sm = P[w];
    __syncwarp();
    for (int i = lane; i < kSm * 8; i += 32) {
        const int g = i / kSm, cc = i - g * kSm, r0 = 4 * g;
        const uint32_t *pc = reinterpret_cast<const uint32_t *>(h + cc * kHP + r0);
        const uint32_t P0 = pc[0], P1 = pc[1], P2 = pc[2], P3 = pc[3], P4 = pc[4];
        const unsigned o0 = __dp2a_lo(P2, kV45, __dp2a_lo(P1, kV23, __dp2a_lo(P0, kV01, kV6 * (P3 & 0xffffu))));
        const unsigned o1 = __dp2a_lo(P3, kW56, __dp2a_lo(P2, kW34, __dp2a_lo(P1, kW12, __dp2a_lo(P0, kW0, 0u))));
        const unsigned o2 = __dp2a_lo(P3, kV45, __dp2a_lo(P2, kV23, __dp2a_lo(P1, kV01, kV6 * (P4 & 0xffffu))));
        const unsigned o3 = __dp2a_lo(P4, kW56, __dp2a_lo(P3, kW34, __dp2a_lo(P2, kW12, __dp2a_lo(P1, kW0, 0u))));
        const unsigned o[4] = {o0, o1, o2, o3};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (r0 + q < kSm) sm[(r0 + q) * kSm + cc] = (uint8_t)((o[q] + 32768u) >> 16);
    }
    // orientation sector: on or left of e_b, strictly right of e_{b+1}
    int bin = 0;
    if (m10 != 0 || m01 != 0) {
        bin = -1;
        if (lane < kBins) {
            const long long mx = m10, my = m01;
            const int b2 = (lane + 1) % kBins;
            const long long c0 = eb[lane][0] * my - eb[lane][1] * mx;
            const long long c1 = eb[b2][0] * my - eb[b2][1] * mx;
            if (c0 >= 0 && c1 < 0) bin = (int)lane;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, bin >= 0);
        bin = bal ? __ffs(bal) - 1 : 0;
    }
    __syncwarp();
    // steered BRIEF: test i = 32 j + lane, word j = ballot
    const int *pat = pattern + bin * kPairs;
    unsigned word = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int pk = __ldg(pat + 32 * j + lane);
        const int px = (int8_t)(pk & 0xff), py = (int8_t)((pk >> 8) & 0xff);
        const int qx = (int8_t)((pk >> 16) & 0xff), qy = (int8_t)((pk >> 24) & 0xff);
        const bool bit = sm[(py + 15) * kSm + px + 15] < sm[(qy + 15) * kSm + qx + 15];
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        if ((int)lane == j) word = bal;
    }
    const int out = pool_off[e] + r;
    unsigned *d = reinterpret_cast<unsigned *>(desc_out + 2LL * out);
    if (lane < 8) d[lane] = word;
    if (lane == 0) {
        asift_keypoint k;
        k.x = (int16_t)x;
        k.y = (int16_t)y;
        k.level = (uint8_t)L.level;
        k.bin = (uint8_t)bin;
        k.view = (uint16_t)v;
        k.r25 = s.r25;
        kp_out[out] = k;
    }
}

// ---------------------------------------------------------------- host side
cudaError_t launch_pyramid(const DevLevel *d_lv, int n, int n_tiles, const int32_t *unit, cudaStream_t s, int grid)
{
    if (n_tiles <= 0) return cudaSuccess;
    const int g = (grid > 0 && grid < n_tiles) ? grid : n_tiles;
    pyramid_kernel<<<g, 256, 0, s>>>(n_tiles, d_lv, n, unit);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mask_rows(const DevLevel *d_lv, int nv, int n_levels, int rows0, int max_h1, int32_t *row_lo,
                             int32_t *row_hi, int32_t *unit, cudaStream_t s)
{
    if (rows0 <= 0 || nv <= 0) return cudaSuccess;
    cudaError_t e0 = cudaMemsetAsync(unit, 0xFF, sizeof(int32_t) * (size_t)nv, s);   // every view unit-convex until a row says not
    if (e0 != cudaSuccess) return e0;
    const int blocks = std::max(1, std::min((rows0 + 7) / 8, 65535));   // a warp per row
    mask_rows_kernel<<<blocks, 256, 0, s>>>(d_lv, nv, rows0, row_lo, row_hi, unit);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n_levels < 2 || max_h1 <= 0) return e;
    const dim3 g((unsigned)((n_levels - 1) * nv), (unsigned)((max_h1 + 255) / 256));
    hull_levels_kernel<<<g, 256, 0, s>>>(d_lv, nv, row_lo, row_hi);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_detect(const DevLevel *d_lv, int n, int n_tiles, int thr, Candidate *cand, int32_t *count,
                          const int32_t *row_lo, const int32_t *row_hi, const int32_t *unit, DetItem *list,
                          int32_t *list_count, cudaStream_t s, int grid)
{
    if (n_tiles <= 0 || n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(list_count, 0, sizeof(int32_t), s);   // the list is rebuilt per launch
    if (e != cudaSuccess) return e;
    det_list_kernel<<<n, 256, 0, s>>>(d_lv, row_lo, row_hi, list, list_count);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int g = grid > 0 ? std::min(grid, n_tiles) : n_tiles;
    detect_kernel<<<g, kDetCols * kDetRowsPar, 0, s>>>(d_lv, list, list_count, thr, cand, count, row_lo, row_hi, unit);
    note_launch();
    return cudaGetLastError();
}

size_t select_smem_bytes() { return (size_t)kSelMax * (sizeof(unsigned long long) + sizeof(unsigned)); }

cudaError_t launch_select(const DevLevel *d_lv, int n, const Candidate *cand, const int32_t *count, int n_features,
                          SlotKp *slots, int32_t *taken, int32_t *status, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = select_smem_bytes();
    const cudaError_t e = ensure_dynamic_smem((const void *)select_kernel, smem);
    if (e != cudaSuccess) return e;
    select_kernel<<<n, kSelThreads, smem, s>>>(d_lv, cand, count, n_features, slots, taken, status);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_pool_scan(const int32_t *taken, int n_views, int n_levels, const int32_t *group_first_view,
                             int n_groups, int n_features, int32_t *pool_off, int32_t *view_count,
                             int32_t *view_off, int32_t *group_total, cudaStream_t s)
{
    if (n_groups <= 0) return cudaSuccess;
    pool_scan_kernel<<<n_groups, 1024, 0, s>>>(taken, n_views, n_levels, group_first_view, n_features, pool_off,
                                               view_count, view_off, group_total);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_orient_brief(const DevLevel *d_lv, int n_views, int n_levels, int n_features, int v_begin,
                                int v_end, const SlotKp *slots, const int32_t *taken, const int32_t *pool_off,
                                const int *pattern, const long long *bins, asift_keypoint *kp, uint4 *desc,
                                cudaStream_t s)
{
    const long long nslots = (long long)(v_end - v_begin) * n_features;
    if (nslots <= 0) return cudaSuccess;
    const int blocks = (int)((nslots + kObWarps - 1) / kObWarps);
    orient_brief_kernel<<<blocks, kObWarps * 32, 0, s>>>(d_lv, n_views, n_levels, n_features, v_begin, v_end, slots,
                                                         taken, pool_off, pattern, bins, kp, desc);
    note_launch();
    return cudaGetLastError();
}

}  // namespace asift
