// common.cuh -- device-side tables and helpers shared by the libasift kernels.
// Internal to the library (the public ABI is include/asift.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "asift.h"

namespace asift {

constexpr int kBorder = 16;       // ORB keypoint border: patch radius 15 + 1
constexpr int kPatchR2 = 225;     // orientation / BRIEF disc x^2 + y^2 <= 15^2
constexpr int kBins = 30;         // 12-degree orientation sectors
constexpr int kPairs = 256;       // rBRIEF-256

// ---------------------------------------------------------------- warp stage
// One view of one source image, as the warp kernel reads it.
struct DevView {
    const float *src;       // source image as fp32, row pitch src_pitch elements
    int32_t src_pitch, W, H;
    int32_t Wr, Hr, Wv, Hv, K;
    int32_t tile_start;     // first linear tile of this view in the launch
    int32_t ntx;            // tiles along x
    int16_t lanes_x;        // canvas columns of a warp's footprint in the rotation step (32, 16 or 8)
    int16_t stage_pitch;    // row pitch (floats) of the staged source box
    int32_t hp;             // floats per view column in filt (>= 2K + 6, a multiple of 4)
    int32_t tw;             // view columns per tile (<= kWarpTW, chosen per view)
    float *filt;            // per view column x: the Gaussian + tilt filter over canvas columns x0-2-K .. x0+3+K
    long long cq, sq, tq;   // Q31 cos, sin, tilt
    long long out_off;      // byte offset of the view in the u8 / mask arenas
    float g[ASIFT_MAX_GAUSS];
};

// Views of one source image whose rotated canvases are identical (the same
// cq, sq, Wr and Hr: the same longitude and scale, tilts differing) share one
// rotation: a tile of the Lanczos-3 warp computes a band of kWarpTH canvas
// rows over one segment of canvas columns once and applies every member
// view's Gaussian + tilt filter to it.
constexpr int kGroupMax = 8;
struct DevRotGroup {
    const float *src;       // source image as fp32 (as DevView::src)
    int32_t src_pitch, W, H, Wr, Hr;
    long long cq, sq;       // Q31 cos / s, sin / s of the members
    int32_t n_views;        // members (indices into the launch's view list)
    int32_t hK;             // largest member K + 3: the strip's halo on either side of a segment
    int32_t nseg, nbands;   // canvas column segments (seg_w columns) and kWarpTH-row bands
    int32_t tile_start;     // first linear tile of this group in the launch
    int16_t lanes_x, stage_pitch;   // rotation step's warp footprint and staging pitch
    int32_t identity;       // 1: cq = 2^31, sq = 0 (phi = 0, s = 1): the canvas is the source itself
    int32_t view[kGroupMax];
};

constexpr int kWarpTW = 64;   // most view columns per warp tile
constexpr int kWarpTH = 16;   // view rows per warp tile
constexpr int kWarpThreads = 256;

// A source image to convert to fp32 (the warp reads fp32 sources).
struct ImageConv {
    const uint8_t *src;
    float *dst;
    int32_t pitch, W, H, dpitch;   // dst rows: dpitch floats, columns >= W zero
};

// Row pitch (floats) of the fp32 source images: a multiple of 4, so that the
// warp kernel stages them with 16-byte copies.
__host__ __device__ inline int src_pitch_of(int W) { return (W + 3) & ~3; }

// ---------------------------------------------------------------- ORB stage
// One (view, pyramid level) as the ORB kernels read it.
struct DevLevel {
    const uint8_t *img;     // level image (pitch W)
    const uint8_t *mask;    // level mask (pitch W)
    uint8_t *img_w;         // writable alias (levels >= 1 are produced by the pyramid kernel)
    uint8_t *mask_w;
    const uint8_t *prev;    // level l-1 image / mask (levels >= 1)
    const uint8_t *prev_mask;
    int32_t W, H, Wp, Hp;   // size, previous level size
    int32_t view, level;
    int32_t quota, qoff;    // keypoint quota of the level and its offset within the view's slots
    int32_t cand_off, cand_cap;   // candidate buffer slice
    int32_t det_tile_start, det_ntx;   // FAST/Harris/NMS tiles
    int32_t pyr_tile_start, pyr_ntx;   // pyramid tiles (levels >= 1)
    int32_t row_off;        // first row of this level in the mask row-hull arrays
    int32_t pad_r;
    // back-projection of a level pixel (x, y) to the source image (Eq. (2)
    // inverted through the level's scale, the tilt and the rotation), one
    // fp64 affine map composed on the host: x_s = bp[0] x + bp[1] y + bp[2],
    // y_s = bp[3] x + bp[4] y + bp[5]
    double bp[6];
};

// Mask row hulls: for every row of every level, the smallest and largest
// column whose mask is 1 (lo > hi when none).  Every pixel outside a row's
// hull has mask 0, so FAST, whose 33 x 33 box needs four mask-valid corners,
// cannot fire at (x, y) unless x - 16 and x + 16 lie in the hulls of rows
// y - 16 and y + 16.  (The views' masks are row-convex, so the hull is the
// valid set itself; the corner test stays the arbiter either way.)
constexpr int32_t kHullEmptyLo = 0x7f7f7f7f;   // byte-fill 0x7f: no column yet
constexpr int32_t kHullEmptyHi = -1;           // byte-fill 0xff

struct Candidate {          // a corner that survived NMS
    long long r25;
    int32_t yx;             // (y << 16) | x
    int32_t pad;
};

struct SlotKp {             // a selected keypoint before orientation / description
    long long r25;
    int32_t yx;             // (y << 16) | x
    int32_t e;              // level entry (relative to the select launch)
};

constexpr int kDetTW = 64, kDetTH = 32;   // FAST tile
constexpr int kPyrTW = 128, kPyrTH = 32;  // pyramid tile (4 columns x 4 rows per thread)

// ---------------------------------------------------------------- differentiable warp
// One view of the differentiable path (image i -> view i).
struct DiffView {
    const float *u;          // source image (pitch W)
    float *ubar;             // its gradient (backward)
    const float *vbar;       // output gradient (backward)
    float *out;              // view (forward)
    const double *param;     // t, phi (deg), tx, ty
    double *pbar;            // dL/d(t, phi, tx, ty) (backward)
    int32_t W, H, Wr, Hr, Wv, Hv, K, tile_start, ntx, tw;   // tw: view columns per tile
};

// A tile of the ORB detection: its level entry and its origin on the level.
struct DetItem {
    int32_t e;
    uint16_t x0, y0;
};

// Per-view constants of the differentiable warp, made once per call on the
// device from the (device-resident) parameters.
struct DiffPrep {
    double dsig_dt;                       // dsigma/dt = 0.8 t / sqrt(t^2 - 1) (0 at t <= 1)
    float c, s;                           // cos, sin of phi
    float sigma, pad;
    float g[ASIFT_MAX_GAUSS];             // normalised Gaussian taps g_0..g_K
    float dg[ASIFT_MAX_GAUSS];            // dg_k / dsigma
};

// ---------------------------------------------------------------- matching
// One brute-force matching problem (query pool vs train pool of one pair),
// with where its results and, for match_pair, its accepted pairs go.
struct MatchProblem {
    const uint4 *q, *t;               // descriptors (2 x uint4 each)
    const int32_t *d_nq, *d_nt;       // device counts (NULL: the capacities are the counts)
    int32_t nq_cap, nt_cap;
    int32_t s_alloc;                  // train slices the partial buffer holds
    int32_t q_off;                    // first query of this problem in a merged launch
    int32_t blk_off, n_blk;           // output blocks of the pair writer
    int32_t cap, pad;                 // accepted-pair capacity
    int *plan;                        // {n_split, chunk} published by the top-2 kernel
    uint2 *part;                      // partial keys [s_alloc][nq_cap]
    asift_match *out;                 // per query
    uint8_t *accept;
    int32_t *n_acc;
    const asift_keypoint *kp1, *kp2;  // pools, for the pair writer
    asift_pair_match *pairs;
    int32_t *d_n;
};

// Launch shapes of the matcher (0 = default).
struct MatchTuning {
    int grid;
    int target_items;
    // failure-path test only (0 = off): the tensor-core matcher's waits give
    // up after stall_ns and its MMA warp first waits on a barrier that nothing
    // arrives at, so that launch ends in ASIFT_ERR_TIMEOUT
    unsigned long long stall_ns = 0;
};

// ---------------------------------------------------------------- helpers
__host__ __device__ inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// The last entry with start <= idx in a monotone table (entries with equal
// starts: the last of them), searched by a whole warp: each round the 32 lanes
// test evenly spaced entries of the remaining range and a ballot keeps the
// highest one that qualifies, so n entries take ceil(log32 n) dependent loads.
// Every lane of the warp must call it with the same arguments.
template <class T, class F>
__device__ inline int find_owner(const T *tab, int n, int idx, F start_of)
{
    const int lane = (int)(threadIdx.x & 31u);
    int lo = 0, hi = n;   // answer in [lo, hi); start_of(tab[lo]) <= idx
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int pos = lo + lane * step;
        const bool ok = pos < hi && start_of(tab[pos]) <= idx;
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        lo += (31 - __clz(b)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Records the first device-side error in the workspace status word.
__device__ inline void set_status(int32_t *status, int32_t code)
{
    if (status) atomicCAS(status, 0, code);
}

}  // namespace asift

// Host-side helpers shared by the API translation units.
namespace asift {
void note_launch(int n = 1);
cudaError_t ensure_dynamic_smem(const void *func, size_t bytes);
int device_sm_count();
}
