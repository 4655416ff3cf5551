/*
 * asift.h -- C ABI of libasift, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of "Feature Point Extraction for Extra-Affine Image"
 * (arXiv 2503.03479): affine view simulation over tilt t and longitude phi
 * (Sec. III-B, Eq. (2)) with a Gaussian anti-alias along the tilt axis and
 * Lanczos-3 resampling (Eq. (3)-(4)), ORB on every view (Sec. III-B: FAST-9 +
 * Harris + NMS on a 1.2 pyramid, intensity-centroid orientation, steered
 * rBRIEF-256), and brute-force Hamming matching with the nearest /
 * second-nearest ratio test over all views of two images (Sec. III-B, IV-C).
 *
 * Problem statement (Sec. III-A, IV-B): given two 8-bit images of one planar
 * scene, return matched point pairs (x1, y1) <-> (x2, y2).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *    pointers owned by the caller.  The library never frees caller memory.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t, NULL = the
 *    legacy default stream).  Host arrays passed in (view tables) are consumed
 *    before the call returns.
 *  - The hot-path calls allocate no device memory: scratch comes from a
 *    caller-provided workspace whose size is returned by the *_workspace_size
 *    queries, 256-byte aligned (as cudaMalloc returns it; asift_views,
 *    match_pair and hamming_match return ASIFT_ERR_ARG otherwise).  Only
 *    asift_ctx_create / asift_plan_create allocate.
 *  - Return value: ASIFT_OK when the work was enqueued; ASIFT_ERR_ARG for a bad
 *    argument (nothing enqueued); ASIFT_ERR_CUDA for a CUDA launch/copy error.
 *    Conditions found on the device while the work runs (a candidate buffer
 *    overflow, a bounded wait that timed out) are written to the int32 status
 *    word at the start of the workspace; read it with asift_read_status after
 *    the stream has progressed past the call.
 *  - No exceptions cross the ABI.  A context is not thread-safe: use one per
 *    host thread.
 */
#ifndef ASIFT_H
#define ASIFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ASIFT_API __attribute__((visibility("default")))
#else
#define ASIFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ASIFT_OK = 0,
    ASIFT_ERR_ARG = -1,      /* invalid argument; nothing was enqueued            */
    ASIFT_ERR_CUDA = -2,     /* CUDA runtime error (launch, copy, no device)      */
    ASIFT_ERR_CAPACITY = -3, /* device-side buffer overflow (status word)         */
    ASIFT_ERR_TIMEOUT = -4,  /* a bounded device wait gave up (status word)       */
    ASIFT_ERR_NOMEM = -5     /* allocation failed in a create call                */
} asift_status;

#define ASIFT_MAX_GAUSS 48   /* Gaussian taps g_0..g_{K}, K < 48 (t <= 11.3)    */
#define ASIFT_MAX_LEVELS 12  /* ORB pyramid levels                              */

/*
 * One simulated view (Eq. (2) with psi = 0, scale s (1 for the views of
 * match_pair; 1 + k ds for the coarse stage), no translation).
 * Geometry, as both this library and any independent check define it:
 *   canvas pixel (i, j) of the Wr x Hr rotated, s-times magnified canvas
 *   takes the source point p = R(phi)^T ((i, j) - c_r) / s + c_s,
 *   c = (size - 1)/2, in Q32 fixed point:
 *     px = cq (2i - Wr + 1) + sq (2j - Hr + 1) + (W - 1) 2^31
 *     py = -sq (2i - Wr + 1) + cq (2j - Hr + 1) + (H - 1) 2^31
 *   view pixel (x', j) samples canvas row j at X = tq (2x' - Wv + 1) + (Wr - 1) 2^31.
 */
typedef struct {
    int32_t k, j;           /* tilt exponent (t = sqrt2^k), longitude index      */
    int32_t W, H;           /* source image size                                  */
    int32_t Wr, Hr;         /* canvas size: ceil(s (W|cos|+H|sin|) - 1e-9), ceil(s (W|sin|+H|cos|) - 1e-9) */
    int32_t Wv, Hv;         /* view size: ceil(Wr / t), Hr                        */
    int32_t K;              /* Gaussian half width ceil(4 sigma)                  */
    int32_t pad0;
    double t, phi_deg;      /* tilt, longitude (degrees)                          */
    double sigma;           /* 0.8 sqrt(t^2 - 1) (0 at t = 1)                     */
    double s;               /* scale: the canvas magnifies the source by s        */
    int64_t cq, sq, tq;     /* rint(cos phi / s 2^31), rint(sin phi / s 2^31), rint(t 2^31) */
    float g[ASIFT_MAX_GAUSS]; /* normalised Gaussian taps g_0..g_K (fp32 of fp64) */
} asift_view_desc;

/* ORB settings (Sec. III-B / IV-C; defaults of the 320x240 configuration). */
typedef struct {
    int32_t n_levels;       /* pyramid levels, scale 1.2 (default 4)             */
    int32_t n_features;     /* keypoints per view (default 500)                  */
    int32_t fast_threshold; /* FAST-9 threshold (default 20)                     */
    int32_t cand_per_mpx;   /* candidate capacity per level, per 10^6 px + 4096 (default 60000) */
} asift_orb_cfg;

/* A keypoint of a view: position in its pyramid level, orientation bin
 * (angle = 12 * bin degrees), Harris response x 25. */
typedef struct {
    int16_t x, y;
    uint8_t level, bin;
    uint16_t view;          /* view index within the call                        */
    int64_t r25;
} asift_keypoint;

/* Result of matching one query descriptor. */
typedef struct {
    int32_t best;           /* index of the nearest train descriptor (-1 if none) */
    uint16_t d1, d2;        /* nearest / second-nearest Hamming distance (257 = none) */
} asift_match;

/* An accepted match, back-projected to source-image pixel coordinates. */
typedef struct {
    float x1, y1, x2, y2;
    int32_t q, t;           /* pool indices in image 1 / image 2                 */
    uint16_t d1, d2;
} asift_pair_match;

typedef struct asift_ctx asift_ctx;

/* Creates a context on the current CUDA device: generates the seeded rBRIEF-256
 * sampling pattern (30 steered copies, ORB [23]) and the orientation sector
 * table on the host and uploads them (allocates ~31 KB).  cfg NULL -> defaults.
 * Errors: ASIFT_ERR_ARG (bad cfg), ASIFT_ERR_NOMEM, ASIFT_ERR_CUDA. */
ASIFT_API asift_status asift_ctx_create(asift_ctx **ctx, const asift_orb_cfg *cfg, uint64_t pattern_seed);
ASIFT_API void asift_ctx_destroy(asift_ctx *ctx);
ASIFT_API asift_status asift_ctx_orb_cfg(const asift_ctx *ctx, asift_orb_cfg *out);
/* Copies the steered pattern (int8 [30][256][4] = {px,py,qx,qy}) to h_out. */
ASIFT_API asift_status asift_ctx_pattern(const asift_ctx *ctx, int8_t *h_out);

/* View table of the sampling rule of Sec. III-B: t = sqrt(2)^k for k = 0..kmax,
 * phi = j 72/t degrees for all j >= 0 with j 72/t < 180 (one view at t = 1).
 * Host only.  Writes min(n, cap) descriptors to h_out (may be NULL) and the
 * total count to *n_views.  Errors: ASIFT_ERR_ARG if H, W < 1 or kmax outside
 * [0, 7]. */
ASIFT_API asift_status asift_view_table(int H, int W, int kmax, asift_view_desc *h_out, int cap, int *n_views);
/* One descriptor for an arbitrary tilt t in [1, 11.4) and longitude phi (deg). */
ASIFT_API asift_status asift_make_view(int H, int W, double t, double phi_deg, asift_view_desc *h_out);
/* The coarse stage's parameter groups (Sec. III-B): the (t, phi) list of
 * asift_view_table with the scale s = 1 + k ds tied to the tilt exponent k
 * (the paper takes ds = 0.5, so s runs 1 .. 3.5 for k <= 5).  ds in [0, 2]. */
ASIFT_API asift_status asift_view_table_scaled(int H, int W, int kmax, double ds, asift_view_desc *h_out, int cap,
                                               int *n_views);
/* One descriptor with a scale s in [1, 8] (asift_make_view is s = 1). */
ASIFT_API asift_status asift_make_view_scaled(int H, int W, double t, double phi_deg, double s,
                                              asift_view_desc *h_out);

/* Host-only copies of the tables a context uploads: the seeded steered rBRIEF
 * pattern (int8 [30][256][4] = {px, py, qx, qy}; SplitMix64 -> Box-Muller
 * N(0, (31/5)^2) rounded ties-to-even inside the radius-15 disc, p != q;
 * rotated by 12 b degrees and rounded half away from zero for b < 15, negated
 * for b >= 15) and the orientation sector boundaries (int64 [30][2], Q30 unit
 * vectors at 12 b - 6 degrees, negated for b >= 15).  ORB [23] steering with a
 * 2 pi / 30 angle discretisation.  Errors: ASIFT_ERR_ARG on NULL. */
ASIFT_API asift_status asift_pattern_table(uint64_t seed, int8_t *h_out);
ASIFT_API asift_status asift_bin_table(int64_t *h_out);

/* Pyramid sizes of a view: W_l = round-half-up(Wv (5/6)^l), exact integers. */
ASIFT_API int asift_level_size(int n0, int level);

/* Bytes of the view arena for n views: sum of Wv*Hv (u8 views), same for masks. */
ASIFT_API int64_t asift_views_bytes(const asift_view_desc *h_views, int n_views);

/*
 * asift_views -- simulate n_views views of one 8-bit image (Eq. (2)-(4)).
 * d_img: H x W uint8 with row pitch `pitch` bytes (>= W).  View v is written
 * at byte offset h_offsets[v] of d_view_u8 and d_mask (Wv*Hv bytes, pitch Wv)
 * and, if d_view_f32 != NULL, at element offset h_offsets[v] of d_view_f32.
 *   canvas C = Lanczos-3 rotation (normalised 6x6 weights, clamp-to-edge taps,
 *              0 outside [-0.5, W-0.5) x [-0.5, H-0.5));
 *   B = Gaussian (taps g) along canvas rows, clamped;
 *   v = Lanczos-3 sample of B at X; u8 = clamp(rint(v)) ties-to-even;
 *   mask = 1 iff canvas columns floor(X) and floor(X)+1 of row j map inside
 *          [0.5, W-1.5] x [0.5, H-1.5].
 * Workspace: asift_views_workspace_size(W, H, n_views).
 */
ASIFT_API size_t asift_views_workspace_size(int H, int W, int n_views);
ASIFT_API asift_status asift_views(asift_ctx *ctx, const uint8_t *d_img, int H, int W, int pitch,
                         const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                         float *d_view_f32, uint8_t *d_view_u8, uint8_t *d_mask,
                         void *d_workspace, size_t ws_bytes, void *stream);

/* asift_views_nearest -- the same views with the coarse stage's
 * nearest-neighbour interpolation (Sec. III-B): canvas C(i, j) = the source
 * pixel at floor(p + 1/2) per axis (Q32; 0 outside the same footprint), B as
 * above, v = B at canvas column clamp(floor(X + 1/2), 0, Wr-1); quantisation,
 * mask, layout, workspace and errors as asift_views. */
ASIFT_API asift_status asift_views_nearest(asift_ctx *ctx, const uint8_t *d_img, int H, int W, int pitch,
                         const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                         float *d_view_f32, uint8_t *d_view_u8, uint8_t *d_mask,
                         void *d_workspace, size_t ws_bytes, void *stream);

/* asift_views_lanczos -- the same views with Lanczos-a resampling, a = 4 for
 * the precise stage's reproduction of the best view (Sec. III-C: an 8 x 8
 * window) or a = 3: Eq. (3)-(4) with 2a normalised taps per axis for the
 * rotation and 2a taps for the tilt, otherwise as asift_views (geometry,
 * background, Gaussian, quantisation, mask, layout, workspace, errors; a
 * outside {3, 4} is ASIFT_ERR_ARG). */
ASIFT_API asift_status asift_views_lanczos(asift_ctx *ctx, int a, const uint8_t *d_img, int H, int W, int pitch,
                                           const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                                           float *d_view_f32, uint8_t *d_view_u8, uint8_t *d_mask,
                                           void *d_workspace, size_t ws_bytes, void *stream);

/*
 * orb_extract -- ORB on n_views views (ORB [23] as used in Sec. III-B).
 * Inputs: views as written by asift_views (d_view_u8 / d_mask at h_offsets).
 * Per view: n_levels pyramid levels (centre-aligned integer bilinear, scale
 * 1.2), FAST-9 (strict, threshold) inside a 16 px border with the four corners
 * of the 33x33 box mask-valid, Harris x25 (Sobel 3x3, 7x7 window, k = 1/25),
 * 3x3 NMS (ties to the raster-first), per-level quota floor(N A_l / sum A)
 * (remainder to level 0), top by (R25 desc, y, x), orientation bin from the
 * centroid moments over the radius-15 disc, steered BRIEF on the level smoothed
 * by [18 34 49 54 49 34 18]/256 per axis.
 * Outputs (capacity n_views * n_features entries): keypoints and 32-byte
 * descriptors in canonical order (view, level, selection order) packed from
 * index 0; d_view_count[v] / d_view_offset[v] give each view's slice (int32).
 * Workspace: orb_workspace_size.  Candidate overflow -> status word
 * ASIFT_ERR_CAPACITY (the view's level keeps its first candidates; result then
 * not defined).
 */
ASIFT_API size_t orb_workspace_size(const asift_ctx *ctx, const asift_view_desc *h_views, int n_views);
ASIFT_API asift_status orb_extract(asift_ctx *ctx, const uint8_t *d_view_u8, const uint8_t *d_mask,
                         const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                         asift_keypoint *d_kp, uint8_t *d_desc, int32_t *d_view_count,
                         int32_t *d_view_offset, int32_t *d_total,
                         void *d_workspace, size_t ws_bytes, void *stream);

/*
 * hamming_match -- brute-force matcher (Sec. III-B) with the ratio test
 * (Sec. IV-C).  For each of nq query descriptors (d_q, nq x 32 bytes, bit i in
 * byte i>>3 at position i&7) over nt train descriptors: best = argmin Hamming
 * distance (lowest index on ties), d1 = its distance, d2 = min over r != best
 * (257 if nt < 2).  Accepted iff nt >= 2 and ratio_den * d1 < ratio_num * d2,
 * exactly in integers (ratio 0.8 = 4/5).  d_out[nq]; d_accept[nq] (uint8, may
 * be NULL); *d_n_accepted (int32, may be NULL).
 * nq and nt may come from the device: if d_nq / d_nt are non-NULL they hold
 * the counts (int32) and nq / nt are only capacities.
 * Workspace: hamming_workspace_size(nq, nt), 256-byte aligned; its first
 * int32 is the status word (cleared by the call, read with asift_read_status).
 */
ASIFT_API size_t hamming_workspace_size(int nq, int nt);
/*
 * Matcher engines (the same results bit for bit; the choice is speed only).
 * ASIFT_MATCH_CUDA_CORES: each thread scans train descriptors with XOR and
 * population counts.  ASIFT_MATCH_TENSOR_CORES: descriptors are expanded to
 * +-1 (fp8 e4m3: +1 for a 0 bit, -1 for a 1 bit) so that the dot product is
 * 256 - 2 x Hamming distance exactly, the dot products of all query / train
 * pairs are computed as a matrix product on the tensor cores (tcgen05, fp32
 * accumulators in tensor memory) and the nearest and second-nearest are
 * selected from the accumulators.  ASIFT_MATCH_AUTO (the default): tensor
 * cores when the device has them (compute capability 10.x), else CUDA cores.
 * asift_ctx_set_match_engine sets the engine of hamming_match and match_pair
 * on this context (ASIFT_ERR_ARG for an unknown value); asking for tensor
 * cores on a device without them makes those calls return ASIFT_ERR_CUDA.
 * asift_ctx_match_engine returns the engine a call would use now (1 or 2).
 * A tensor-core launch that waits more than 4 s on one of its own pipeline
 * stages gives up and records ASIFT_ERR_TIMEOUT in the workspace status word.
 */
#define ASIFT_MATCH_AUTO 0
#define ASIFT_MATCH_CUDA_CORES 1
#define ASIFT_MATCH_TENSOR_CORES 2
ASIFT_API asift_status asift_ctx_set_match_engine(asift_ctx *ctx, int engine);
ASIFT_API int asift_ctx_match_engine(const asift_ctx *ctx);

/*
 * Failure-path test hooks.  The paper has no counterpart: these exist so that
 * tests can drive the device-side error paths without a GPU fault.  Each hook
 * holds until it is set again; value 0 turns it off.  Setting a hook drops
 * match_pair's cached layouts of this context (the capacities change).
 *  ASIFT_HOOK_CAND_CAP: every pyramid level's candidate list holds `value`
 *    corners (1 .. 2^30, at most the level's pixel count) instead of 4096 +
 *    cand_per_mpx x pixels / 10^6; a level with more NMS survivors sets
 *    ASIFT_ERR_CAPACITY in the status word (orb_extract, match_pair, plans
 *    created while it is set).
 *  ASIFT_HOOK_MATCH_STALL: value = a wait limit in ns (1000 .. 4e9).  Every
 *    tensor-core matcher launch of this context (hamming_match, match_pair)
 *    bounds its waits by `value` instead of 4 s, and its MMA warp first waits
 *    on a barrier that nothing arrives at: that wait runs out, the launch
 *    records ASIFT_ERR_TIMEOUT, lets its copies land, frees its tensor
 *    memory and returns; its match results are then undefined.
 * Errors: ASIFT_ERR_ARG for a NULL context, an unknown hook or a value out of
 * range.
 */
#define ASIFT_HOOK_CAND_CAP 1
#define ASIFT_HOOK_MATCH_STALL 2
ASIFT_API asift_status asift_ctx_set_test_hook(asift_ctx *ctx, int hook, int64_t value);
ASIFT_API asift_status hamming_match(asift_ctx *ctx, const uint8_t *d_q, int nq, const int32_t *d_nq,
                           const uint8_t *d_t, int nt, const int32_t *d_nt,
                           int ratio_num, int ratio_den, asift_match *d_out, uint8_t *d_accept,
                           int32_t *d_n_accepted, void *d_workspace, size_t ws_bytes, void *stream);

/*
 * hamming_match_noalloc -- the same matcher as hamming_match (same results, bit
 * for bit) for callers that cannot allocate device memory: code handed only its
 * input and output buffers by a host framework that owns all device memory and
 * offers no workspace, and latency-bound loops that forbid cudaMalloc/cudaFree
 * after start-up because those calls can synchronise the device and take
 * unbounded time.  This paper-independent convenience has no counterpart in
 * the paper.
 * It takes no context and no workspace: its scratch (the per-slice partial
 * nearest / second-nearest keys) is a fixed device array of
 * ASIFT_NOALLOC_SCRATCH_BYTES that the library declares at file scope, so every
 * GPU that loads the library holds those bytes until the process exits.
 * Limits: nq <= ASIFT_NOALLOC_MAX_QUERIES and nt <= 8388607; larger sizes return
 * ASIFT_ERR_ARG with nothing enqueued.  The first call in each CUDA context
 * (the device current at the call) looks up the array's device address, a
 * host-side query that allocates nothing; make that first call before any
 * stream capture on that device.  After cudaDeviceReset the device has a new
 * context and the next call looks the address up again.  Every call uses the same
 * array and leaves its contents behind (nothing in it needs to start at zero:
 * each call writes every entry it reads), so calls whose work overlaps on the
 * GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  Arguments otherwise as hamming_match.
 */
#define ASIFT_NOALLOC_SCRATCH_BYTES (8u << 20)
#define ASIFT_NOALLOC_MAX_QUERIES 1000000
ASIFT_API asift_status hamming_match_noalloc(const uint8_t *d_q, int nq, const int32_t *d_nq, const uint8_t *d_t,
                                             int nt, const int32_t *d_nt, int ratio_num, int ratio_den,
                                             asift_match *d_out, uint8_t *d_accept, int32_t *d_n_accepted,
                                             void *stream);

/* View-set configuration of match_pair. */
/* Interpolation of the simulated views. */
#define ASIFT_INTERP_LANCZOS3 0
#define ASIFT_INTERP_NEAREST 1

typedef struct {
    int32_t kmax;           /* t = sqrt2^k, k = 0..kmax (default 5)             */
    int32_t ratio_num, ratio_den; /* ratio test (default 4/5)                   */
    int32_t per_view;       /* 1 = launch every stage once per view (the plain
                               per-view form); 0 = one launch per stage over all
                               views of both images                            */
    int32_t coarse;         /* 1 = the coarse stage of Sec. III-B: image 1 (the
                               reference) takes the parameter groups of
                               asift_view_table_scaled(kmax, ds), image 2 (the
                               target) its single unwarped view; 0 = both images
                               the views of asift_view_table(kmax)             */
    int32_t interp;         /* ASIFT_INTERP_LANCZOS3 (default) or
                               ASIFT_INTERP_NEAREST, the coarse stage's
                               nearest-neighbour views (asift_views_nearest) */
    double ds;              /* scale step of the coarse stage (default 0.5)     */
} asift_pair_cfg;

/*
 * match_pair -- the whole hot path for one image pair: the views of both
 * images (sampling rule of Sec. III-B), ORB on every view, pooling of each
 * image's keypoints in canonical order, brute-force matching of pool 1 against
 * pool 2 with the ratio test, and back-projection of the accepted pairs to
 * source-image coordinates.  d_out receives up to `cap` accepted pairs in
 * query order; *d_n (int32) their count (may exceed cap: then the status word
 * is ASIFT_ERR_CAPACITY).  Workspace: match_pair_workspace_size.
 */
ASIFT_API size_t match_pair_workspace_size(const asift_ctx *ctx, int H1, int W1, int H2, int W2,
                                 const asift_pair_cfg *cfg);
ASIFT_API asift_status match_pair(asift_ctx *ctx, const uint8_t *d_img1, int H1, int W1, int pitch1,
                        const uint8_t *d_img2, int H2, int W2, int pitch2,
                        const asift_pair_cfg *cfg, asift_pair_match *d_out, int cap, int32_t *d_n,
                        void *d_workspace, size_t ws_bytes, void *stream);

/*
 * Batched form: all views of many image pairs (uneven sizes) in one launch per
 * stage, captured once in a CUDA graph and replayed.  asift_plan_create
 * builds the view / level / matching tables of every pair, allocates the
 * plan's device workspace and output buffers (the only allocation), uploads
 * the tables, runs the sequence once uncaptured to validate it, and captures
 * it in a CUDA graph (use_graph != 0).  The image pointers are fixed at
 * creation: update the images in place between runs.  asift_plan_run replays
 * the graph (or relaunches the sequence) on `stream`; results are bit-identical
 * to match_pair on each pair.  Errors: ASIFT_ERR_ARG, ASIFT_ERR_NOMEM,
 * ASIFT_ERR_CUDA.
 */
typedef struct {
    const uint8_t *d_img1;
    int32_t H1, W1, pitch1;
    const uint8_t *d_img2;
    int32_t H2, W2, pitch2;
} asift_pair_desc;

/* Launch shapes of the batched stages (0 = one CTA per tile / the default).
 * A positive grid makes the stage's kernel persistent over its tile list.
 * The detection runs over the list of tiles that can hold corners.
 * warp_seg is the tile shape of the view simulation: the canvas columns a
 * tile rotates once and filters for every view sharing that rotation
 * (0 = the default 576; 64 .. 1024; wider tiles recompute less of the
 * Gaussian's halo but hold more shared memory, so fewer fit on an SM). */
typedef struct {
    int32_t warp_grid, pyramid_grid, detect_grid, match_grid, match_target_items;
    int32_t match_engine;   /* ASIFT_MATCH_*; ASIFT_MATCH_AUTO = the context's engine */
    int32_t warp_seg;       /* canvas columns per view-simulation tile (0 = 576) */
} asift_tuning;

typedef struct asift_plan asift_plan;
ASIFT_API asift_status asift_plan_create(asift_ctx *ctx, const asift_pair_desc *h_pairs, int n_pairs,
                                         const asift_pair_cfg *cfg, const asift_tuning *tuning, int use_graph,
                                         asift_plan **out);
ASIFT_API asift_status asift_plan_run(asift_plan *plan, void *stream);
/* Device pointers of pair i's accepted matches, their capacity and count. */
ASIFT_API asift_status asift_plan_pairs(const asift_plan *plan, int i, asift_pair_match **d_pairs, int *cap,
                                        int32_t **d_n);
/* match_pair_view_counts for pair i of the plan's last run (on `stream`, in
 * order after asift_plan_run): accepted matches per image-1 view of pair i
 * (its view table order) and the view with the most. */
ASIFT_API asift_status asift_plan_view_counts(const asift_plan *plan, int i, int32_t *d_counts, int n_counts,
                                              int32_t *d_best, void *stream);
/* The plan's workspace (status word first) and the pooled keypoint counts
 * (int32 [2 n_pairs]: image 1, image 2 of each pair). */
ASIFT_API asift_status asift_plan_workspace(const asift_plan *plan, void **d_workspace, int32_t **d_pool_counts);
ASIFT_API asift_status asift_plan_set_tuning(asift_plan *plan, const asift_tuning *tuning);
ASIFT_API asift_status asift_plan_get_tuning(const asift_plan *plan, asift_tuning *out);
/* Autotuner: times candidate launch shapes of each stage (coordinate descent,
 * `reps` graph replays per candidate, CUDA events on the plan's stream), keeps
 * the fastest, re-captures the graph and returns the choice in *out. */
ASIFT_API asift_status asift_plan_autotune(asift_plan *plan, int reps, asift_tuning *out);
ASIFT_API void asift_plan_destroy(asift_plan *plan);

/*
 * Differentiable warp (the photometric refinement of a simulated view's
 * parameters).  n images of H x W fp32 (image i at offset i*H*W of d_u), one
 * view each, with device parameters d_params[4 i ..] = (t, phi in degrees, tx,
 * ty) and fixed host shapes (asift_warp_shape_for: the canvas / view sizes of
 * (t0, phi0) and K = ceil(4 * 0.8 sqrt(t_max^2 - 1))).  The map is Eq. (2)-(4)
 * with p = R(phi)^T (q - c_r) + c_s + (tx, ty), every Lanczos tap clamped to
 * the image (no zero background) and sigma = 0.8 sqrt(t^2 - 1) with the fixed
 * K, so it is continuously differentiable in (u, t, phi, tx, ty).
 * asift_warp_fwd writes view i at element offset h_voff[i] of d_v (pitch Wv).
 * asift_warp_bwd takes the output gradient d_vbar (same layout) and writes the
 * image gradient d_ubar (n x H x W, overwritten) and d_pbar[4 i ..] =
 * dL/d(t, phi [per degree], tx, ty) (overwritten); the canvas and its blur are
 * recomputed, nothing is kept from the forward.  d_ubar may be NULL: then only
 * the parameter gradients are computed (the image gradient's scatter is
 * skipped, as photometric descent of the parameters needs).  A t above t_max
 * sets the status word to ASIFT_ERR_CAPACITY.  Workspace:
 * asift_warp_workspace_size(n).
 */
typedef struct {
    int32_t Wr, Hr, Wv, Hv, K, pad;
} asift_warp_shape;
ASIFT_API asift_status asift_warp_shape_for(int H, int W, double t0, double phi0, double t_max,
                                            asift_warp_shape *out);
ASIFT_API size_t asift_warp_workspace_size(int n);
ASIFT_API asift_status asift_warp_fwd(asift_ctx *ctx, const float *d_u, int H, int W, int n, const double *d_params,
                                      const asift_warp_shape *h_shapes, double t_max, float *d_v,
                                      const int64_t *h_voff, void *d_workspace, size_t ws_bytes, void *stream);
ASIFT_API asift_status asift_warp_bwd(asift_ctx *ctx, const float *d_u, int H, int W, int n, const double *d_params,
                                      const asift_warp_shape *h_shapes, double t_max, const float *d_vbar,
                                      const int64_t *h_voff, float *d_ubar, double *d_pbar, void *d_workspace,
                                      size_t ws_bytes, void *stream);

/*
 * Photometric descent of the view parameters (the refinement of the best
 * simulated view's tilt and rotation; the paper has no descent, the
 * configuration asks for one).
 * asift_warp_loss: per view i (layout of asift_warp_fwd: h_shapes, h_voff),
 * d_loss[i] = the mean over its pixels of (d_v - d_target)^2 (fp32 squares,
 * fp64 sums; overwritten) and, when d_vbar is non-NULL, the gradient of the
 * summed losses, d_vbar = 2 (d_v - d_target) / (Wv Hv) (fp32, same layout).
 * Workspace: asift_warp_workspace_size(n).
 * asift_warp_adam: one Adam step on d_params (n x (t, phi, tx, ty), fp64)
 * with the gradient d_grad (as asift_warp_bwd writes it) and the moment
 * buffers d_m, d_v (n x 4 doubles, zero before step 0): b1 = 0.9, b2 = 0.999,
 * eps = 1e-12, step sizes h_lr[4] x decay^step, bias correction with
 * step + 1; a view whose gradient is not finite takes a zero gradient (its
 * moments still move it); t is clamped to [t_lo, t_hi].  Errors: ASIFT_ERR_ARG for NULL buffers, n < 1,
 * step < 0, decay <= 0 or a t range outside [1, 11.4).
 */
ASIFT_API asift_status asift_warp_loss(asift_ctx *ctx, int n, const asift_warp_shape *h_shapes, const int64_t *h_voff,
                                       const float *d_v, const float *d_target, double *d_loss, float *d_vbar,
                                       void *d_workspace, size_t ws_bytes, void *stream);
ASIFT_API asift_status asift_warp_adam(asift_ctx *ctx, int n, double *d_params, const double *d_grad, double *d_m,
                                       double *d_v, int step, const double *h_lr, double decay, double t_lo,
                                       double t_hi, void *stream);

/* Debug view into match_pair's workspace after a call: device pointers to the
 * pooled keypoints / descriptors / per-query matches of each image and the
 * host view tables used.  Any output pointer may be NULL. */
ASIFT_API asift_status match_pair_inspect(const asift_ctx *ctx, int H1, int W1, int H2, int W2,
                                const asift_pair_cfg *cfg, void *d_workspace,
                                asift_keypoint **d_kp1, uint8_t **d_desc1, int32_t **d_n1,
                                asift_keypoint **d_kp2, uint8_t **d_desc2, int32_t **d_n2,
                                asift_match **d_match);

/*
 * asift_sift -- SIFT (Lowe 2004) keypoints and descriptors of one 8-bit image,
 * the detector of the precise stage (Sec. III-C), fp32: the image / 255
 * doubled (centre-aligned bilinear), blurred to sigma0 = 1.6 from an assumed
 * 2 x 0.5; S = 3 intervals per octave, floor(log2 min(2W, 2H)) - 3 octaves
 * (at most 12), each started from image S of the previous subsampled by 2;
 * strict 26-neighbour DoG extrema 5 px from the border with |D| > 0.5 x 0.04 /
 * S; quadratic refinement (at most 5 moves), |D^| >= 0.04 / S, edge ratio
 * tr^2 / det < 11^2 / 10; 36-bin orientation histograms (window 1.5 sigma,
 * radius 3 x 1.5 sigma, [1 4 6 4 1] / 16 smoothing, every peak within 80% of
 * the highest, parabolic refinement; angle of the gradient atan2(gy, gx) in
 * degrees, y down); 4 x 4 x 8 descriptors over the window rotated to the
 * orientation (bins 3 sigma wide, trilinear spreading, Gaussian weight of
 * half the window), unit-normalised, clamped at 0.2, renormalised.
 * d_kp[max_kp] and d_desc[max_kp x 128] (device) receive the keypoints in
 * an unspecified order; *d_n (device) the number found: when it exceeds
 * max_kp, which max_kp are written is unspecified (refined extrema are held
 * up to max(max_kp, W H / 2 + 1024) before their orientations).  Descriptor
 * histograms accumulate with shared-memory atomics, so their last bits can
 * differ between runs; keypoints do not.  Workspace:
 * asift_sift_workspace_size(H, W, max_kp) bytes, 256-byte aligned.  Errors:
 * ASIFT_ERR_ARG for NULL or misaligned buffers, W or H below 16 or above
 * 16384, max_kp outside [1, 2^20].
 */
typedef struct {
    float x, y;             /* original image coordinates                      */
    float sigma;            /* scale in original image pixels                  */
    float angle;            /* degrees, [0, 360)                               */
    float response;         /* |D| at the refined extremum                     */
    int32_t octave, layer;
    float xo, yo, so;       /* position and scale in the octave's pixels       */
    int32_t pad[2];
} asift_sift_kp;
ASIFT_API size_t asift_sift_workspace_size(int H, int W, int max_kp);
ASIFT_API asift_status asift_sift(asift_ctx *ctx, const uint8_t *d_img, int H, int W, int pitch, int max_kp,
                                  asift_sift_kp *d_kp, float *d_desc, int32_t *d_n, void *d_workspace,
                                  size_t ws_bytes, void *stream);

/*
 * asift_sift_match -- brute-force L2 matching of SIFT descriptors with the
 * ratio test: the matching of the precise stage (Sec. III-C, SIFT on the
 * reproduced best view against the target) and the match list that Eq. (1)
 * takes (Sec. III-A).  For each of the queries d_q (nq x 128 fp32, as
 * asift_sift writes them) over the trains d_t (nt x 128): the squared
 * distance is the fp32 sum over c = 0..127, in that order, of e_c^2 with
 * e_c = q_c - t_c rounded to fp32, each term added by one fused multiply-add
 * (the decisions are taken in fp32 in this fixed order, so any implementation
 * of it gives the same bits); best = the lowest index among the smallest
 * distances, d2 = the second smallest (d2 = d1 on a tie; INFINITY when there
 * is none); accepted iff nt >= 2 and d1 < r2 * d2 in fp32 with r2 =
 * (float)(ratio * ratio) (Lowe's ratio test on distances; 0.8 by default).
 * d_out[nq] (asift_l2_match) receives every query's result.  With keypoints
 * d_kq / d_kt (asift_sift_kp, may be NULL) and d_n_pairs non-NULL, the
 * accepted queries are written in query order to d_pairs (up to cap) as
 * asift_pair_match: x1, y1 = d_kq[q], x2, y2 = d_kt[best], d1 / d2 = the L2
 * distances at the scale of integer SIFT descriptors (512 sqrt(d), rounded),
 * which is the scale Eq. (1)'s weight 1 - (Des_i + Des_i+1) / 1000 is written
 * for; *d_n_pairs = their count (above cap: status ASIFT_ERR_CAPACITY).
 * nq / nt may come from the device (d_nq / d_nt, clamped to nq / nt, e.g.
 * asift_sift's count).  Workspace: asift_sift_match_workspace_size(nq, nt),
 * 256-byte aligned, status word first.  Errors: ASIFT_ERR_ARG for NULL or
 * misaligned buffers, nq or nt outside [0, 2^22], a ratio outside (0, 1].
 */
typedef struct {
    int32_t best;           /* nearest train descriptor (-1 if none)              */
    float d1, d2;           /* nearest / second-nearest squared distance (fp32)   */
} asift_l2_match;
ASIFT_API size_t asift_sift_match_workspace_size(int nq, int nt);
ASIFT_API asift_status asift_sift_match(asift_ctx *ctx, const float *d_q, int nq, const int32_t *d_nq, const float *d_t,
                                        int nt, const int32_t *d_nt, double ratio, const asift_sift_kp *d_kq,
                                        const asift_sift_kp *d_kt, asift_l2_match *d_out, asift_pair_match *d_pairs,
                                        int cap, int32_t *d_n_pairs, void *d_workspace, size_t ws_bytes,
                                        void *stream);

/* Base-image selection, Eq. (1) (Sec. III-A): the scaling coefficient from
 * image 1 to image 2 over the pairs d_pairs[0 .. min(*d_n, cap) - 1] in list
 * order,
 *   f = sum_{i + 1 < n} (|a_i+1 - a_i| - |b_i+1 - b_i|) (1 - (Des_i + Des_i+1) / 1000)
 * with a_i = (x1, y1), b_i = (x2, y2) and Des_i = d1 (the pair's descriptor
 * distance: the SIFT L2 distance at integer-descriptor scale for the pairs of
 * asift_sift_match, as the paper defines it, or the rBRIEF Hamming distance
 * for those of match_pair), in fp64,
 * summed in a fixed order.  f > 0: the scene appears larger in image 1.
 * Computing f1 on image 1 -> 2's pairs and f2 on image 2 -> 1's, image 1 is
 * the reference when f1 > f2.  *d_f (device) is written on `stream`.
 * Workspace: asift_scale_coefficient_workspace_size(cap) bytes, 256-byte
 * aligned.  d_n may point into another call's output (e.g. n_unique of an
 * asift_eval_result, with its kept pairs as d_pairs). */
ASIFT_API size_t asift_scale_coefficient_workspace_size(int cap);
ASIFT_API asift_status asift_scale_coefficient(asift_ctx *ctx, const asift_pair_match *d_pairs, const int32_t *d_n,
                                               int cap, double *d_f, void *d_workspace, size_t ws_bytes,
                                               void *stream);

/* Coarse stage, best-parameter selection (Sec. III-B): after a match_pair call
 * on d_workspace with the same sizes and configuration, d_counts[v] (v = 0 ..
 * n1 - 1, n1 = the number of image 1's views, in table order) receives the
 * number of accepted matches whose image-1 keypoint was detected in view v,
 * and *d_best (when d_best is not NULL) the view with the most, the lowest v
 * among equal counts.  With cfg->coarse = 1 the views are the parameter groups
 * (t, phi, s) of asift_view_table_scaled and image 2 is the unwarped target, so
 * d_counts[*d_best] names the best parameter group.  Device outputs, written
 * on `stream` in order after the match_pair launches; the caller owns them.
 * Errors: ASIFT_ERR_ARG for NULL pointers, a per-view configuration, n_counts
 * below n1, or n1 above 8192. */
ASIFT_API asift_status match_pair_view_counts(asift_ctx *ctx, int H1, int W1, int H2, int W2,
                                              const asift_pair_cfg *cfg, void *d_workspace, int32_t *d_counts,
                                              int n_counts, int32_t *d_best, void *stream);

/*
 * Evaluation of the accepted pairs of a match_pair call (Sec. III-C, Sec. IV-B):
 *   1. duplicate removal in original coordinates: pair i is dropped when an
 *      earlier pair has the same nearest pixels floor(c + 1/2) (fp32) of all
 *      four coordinates (x1, y1, x2, y2) -- several views can detect the same
 *      correspondence; the kept pairs are written, in order, to d_unique;
 *   2. precision (Eq. (5)-(6)): with a true homography h_H_true (host, 9
 *      doubles, row-major, image 1 -> image 2), r_num = the kept pairs with
 *      |H (x1, y1) - (x2, y2)|^2 <= th_sq (th_sq = 3 for the paper's sqrt 3);
 *      precision = r_num / n_unique;
 *   3. RANSAC [28]: hypothesis h fits a homography (h8 = 1, Gaussian
 *      elimination with partial pivoting on the eight DLT equations) to the
 *      kept pairs d_rnd[4h + k] mod n_unique (k = 0..3; d_rnd: device uint32,
 *      4 n_hyp, the caller's random numbers); a repeated pair or a pivot at
 *      most 1e-10 times the system's largest |entry| leaves it out (count -1);
 *      its count is the kept pairs with squared reprojection error <=
 *      ransac_th_sq; the best has the largest count, the lowest h on ties;
 *   4. inliers (Eq. (7)): d_inlier[i] (cap bytes, may be NULL) = kept pair i
 *      is within the threshold of the best H; n_inliers = their number,
 *      inlier ratio = n_inliers / n_unique.
 * Every fp64 step is one correctly rounded operation in the order written
 * above (reprojection: ((h0 x + h1 y) + h2) / ((h6 x + h7 y) + h8) - x2, ...).
 * d_pairs / d_n: match_pair's output (count clamped to cap).  d_hyp_counts
 * (n_hyp int32, may be NULL) receives the per-hypothesis counts.  Results go
 * to the device struct d_result, in stream order.  Workspace:
 * asift_eval_workspace_size(cap, n_hyp) bytes, 256-byte aligned.
 * Errors: ASIFT_ERR_ARG for NULL or misaligned buffers, cap outside
 * [0, 2^26], n_hyp outside [0, 2^20] or negative thresholds.
 */
typedef struct {
    int32_t n_pairs;        /* accepted pairs read: min(*d_n, cap)               */
    int32_t n_unique;       /* Pt_Num: pairs left after duplicate removal        */
    int32_t r_num;          /* R_Num of Eq. (5)-(6); -1 without a true H         */
    int32_t best_hyp;       /* best RANSAC hypothesis; -1 if none fits           */
    int32_t n_inliers;      /* In_Num of Eq. (7)                                 */
    int32_t status;         /* ASIFT_OK (ASIFT_ERR_CAPACITY: table overflow)     */
    double ransac_th_sq;    /* the squared RANSAC threshold used                 */
    double H[9];            /* the best hypothesis, row-major; zeros if none     */
} asift_eval_result;
ASIFT_API size_t asift_eval_workspace_size(int cap, int n_hyp);
ASIFT_API asift_status asift_eval_pairs(asift_ctx *ctx, const asift_pair_match *d_pairs, const int32_t *d_n, int cap,
                                        const double *h_H_true, double th_sq, const uint32_t *d_rnd, int n_hyp,
                                        double ransac_th_sq, asift_pair_match *d_unique, uint8_t *d_inlier,
                                        int32_t *d_hyp_counts, asift_eval_result *d_result, void *d_workspace,
                                        size_t ws_bytes, void *stream);

/* asift_eval_pairs for every pair of the plan's last run, one launch per
 * stage over all pairs: h_H_true holds 9 doubles per pair (or NULL: no
 * precision), the n_hyp hypotheses' random numbers d_rnd are shared by all
 * pairs.  Outputs (kept pairs, inlier mask, per-hypothesis counts, result)
 * live in d_workspace (asift_plan_eval_workspace_size(plan, n_hyp) bytes,
 * 256-byte aligned); asift_plan_eval_outputs returns pair i's (any output
 * pointer may be NULL).  Results equal asift_eval_pairs on each pair. */
ASIFT_API size_t asift_plan_eval_workspace_size(const asift_plan *plan, int n_hyp);
ASIFT_API asift_status asift_plan_eval(asift_plan *plan, const double *h_H_true, double th_sq, const uint32_t *d_rnd,
                                       int n_hyp, double ransac_th_sq, void *d_workspace, size_t ws_bytes,
                                       void *stream);
ASIFT_API asift_status asift_plan_eval_outputs(const asift_plan *plan, void *d_workspace, int n_hyp, int i,
                                               asift_pair_match **d_unique, uint8_t **d_inlier,
                                               int32_t **d_hyp_counts, asift_eval_result **d_result);

/* Synchronises `stream` and copies the status word at the start of a
 * workspace to *h_status (ASIFT_OK, ASIFT_ERR_CAPACITY or ASIFT_ERR_TIMEOUT);
 * clears it when clear != 0. */
ASIFT_API asift_status asift_read_status(void *d_workspace, int clear, int32_t *h_status, void *stream);

/* Stage timing of match_pair with CUDA events on the call's stream.  Stages:
 * 0 input upload + conversion, 1 warp, 2 pyramid, 3 FAST/Harris/NMS,
 * 4 top-N selection, 5 pool offsets + orientation + BRIEF, 6 Hamming match,
 * 7 accepted-pair output.  Enabling creates the events (no device memory).
 * asift_profile_read synchronises on the last recorded event and writes the
 * milliseconds of each stage of the most recent match_pair to h_ms[0..n). */
#define ASIFT_PROF_STAGES 8
ASIFT_API asift_status asift_profile_enable(asift_ctx *ctx, int on);
ASIFT_API asift_status asift_profile_read(asift_ctx *ctx, float *h_ms, int n);

/* Number of kernels this library has launched in the calling process. */
ASIFT_API int64_t asift_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* ASIFT_H */
