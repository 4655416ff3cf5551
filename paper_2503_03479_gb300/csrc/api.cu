// api.cu -- the C ABI of libasift (include/asift.h): contexts, workspace
// layouts, and the launch sequences of asift_views, orb_extract,
// hamming_match and match_pair.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace asift {

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------- workspace bump allocator
struct Bump {
    char *base;
    size_t off = 0;
    explicit Bump(void *b) : base(static_cast<char *>(b)) {}
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * count;
        return p;
    }
};

// ---------------------------------------------------------------- level tables
struct LevelTables {
    std::vector<DevLevel> lv;     // level-major: index l * n_views + v
    std::vector<int> pyr_tiles;   // tiles of the pyramid launch of each level
    int det_tiles = 0;
    long long cand_total = 0;
    long long arena_bytes = 0;    // bytes of the levels kept in the workspace arena
};

static int cand_capacity(const asift_orb_cfg &cfg, int W, int H)
{
    const long long c = 4096 + (long long)cfg.cand_per_mpx * W * H / 1000000;
    return (int)std::min<long long>(c, (long long)W * H);
}

static int level_quota(const asift_orb_cfg &cfg, const int *Ws, const int *Hs, int l)
{
    long long S = 0, used = 0;
    for (int i = 0; i < cfg.n_levels; ++i) S += (long long)Ws[i] * Hs[i];
    for (int i = 0; i < cfg.n_levels; ++i) used += (long long)cfg.n_features * Ws[i] * Hs[i] / S;
    const long long q = (long long)cfg.n_features * Ws[l] * Hs[l] / S;
    return (int)(l == 0 ? q + (cfg.n_features - used) : q);
}

// Level tables of n views.  Level 0 of view v is (l0_img[v], l0_mask[v]) when
// given, otherwise it lives in the arena like the other levels.  per_view:
// every tile_start is 0 (each entry is launched on its own).
static void build_levels(const asift_orb_cfg &cfg, const asift_view_desc *views, int nv,
                         const uint8_t *const *l0_img, const uint8_t *const *l0_mask, uint8_t *arena_u8,
                         uint8_t *arena_mask, bool per_view, LevelTables &T)
{
    const int L = cfg.n_levels;
    T.lv.assign((size_t)L * nv, DevLevel{});
    T.pyr_tiles.assign(L, 0);
    T.det_tiles = 0;
    T.cand_total = 0;
    T.arena_bytes = 0;
    std::vector<long long> level_off((size_t)L * nv, -1);
    // arena layout: view-major, levels contiguous
    for (int v = 0; v < nv; ++v)
        for (int l = (l0_img ? 1 : 0); l < L; ++l) {
            const int W = level_size(views[v].Wv, l), H = level_size(views[v].Hv, l);
            level_off[(size_t)l * nv + v] = T.arena_bytes;
            T.arena_bytes += ((long long)W * H + 15) & ~15LL;
        }
    for (int l = 0; l < L; ++l) {
        for (int v = 0; v < nv; ++v) {
            DevLevel &d = T.lv[(size_t)l * nv + v];
            int Ws[ASIFT_MAX_LEVELS], Hs[ASIFT_MAX_LEVELS];
            for (int i = 0; i < L; ++i) {
                Ws[i] = level_size(views[v].Wv, i);
                Hs[i] = level_size(views[v].Hv, i);
            }
            d.W = Ws[l];
            d.H = Hs[l];
            d.Wp = l ? Ws[l - 1] : 0;
            d.Hp = l ? Hs[l - 1] : 0;
            d.view = v;
            d.level = l;
            d.quota = level_quota(cfg, Ws, Hs, l);
            int qoff = 0;
            for (int i = 0; i < l; ++i) qoff += level_quota(cfg, Ws, Hs, i);
            d.qoff = qoff;
            const long long off = level_off[(size_t)l * nv + v];
            if (l == 0 && l0_img) {
                d.img = l0_img[v];
                d.mask = l0_mask[v];
                d.img_w = nullptr;
                d.mask_w = nullptr;
            } else {
                d.img_w = arena_u8 ? arena_u8 + off : nullptr;
                d.mask_w = arena_mask ? arena_mask + off : nullptr;
                d.img = d.img_w;
                d.mask = d.mask_w;
            }
            if (l > 0) {
                const DevLevel &p = T.lv[(size_t)(l - 1) * nv + v];
                d.prev = p.img;
                d.prev_mask = p.mask;
            }
            d.cand_cap = cand_capacity(cfg, d.W, d.H);
            d.cand_off = (int)T.cand_total;
            T.cand_total += d.cand_cap;
            d.det_ntx = (d.W + kDetTW - 1) / kDetTW;
            const int det = d.det_ntx * ((d.H + kDetTH - 1) / kDetTH);
            d.det_tile_start = per_view ? 0 : T.det_tiles;
            T.det_tiles += det;
            d.pyr_ntx = (d.W + kPyrTW - 1) / kPyrTW;
            const int pyr = d.pyr_ntx * ((d.H + kPyrTH - 1) / kPyrTH);
            d.pyr_tile_start = per_view ? 0 : T.pyr_tiles[l];
            T.pyr_tiles[l] += pyr;
        }
    }
}

static int det_tiles_of(const DevLevel &d) { return d.det_ntx * ((d.H + kDetTH - 1) / kDetTH); }
static int pyr_tiles_of(const DevLevel &d) { return d.pyr_ntx * ((d.H + kPyrTH - 1) / kPyrTH); }

// View tables for the warp kernel.
static void build_views(const asift_view_desc *h, int nv, const float *const *src, const int *src_pitch,
                        const int64_t *out_off, bool per_view, std::vector<DevView> &out, int *n_tiles,
                        int *cw_max, int *bw_max)
{
    out.assign(nv, DevView{});
    int tiles = 0, cwm = 1, bwm = 1;
    for (int v = 0; v < nv; ++v) {
        const asift_view_desc &a = h[v];
        DevView &d = out[v];
        d.src = src[v];
        d.src_pitch = src_pitch[v];
        d.W = a.W;
        d.H = a.H;
        d.Wr = a.Wr;
        d.Hr = a.Hr;
        d.Wv = a.Wv;
        d.Hv = a.Hv;
        d.K = a.K;
        d.cq = a.cq;
        d.sq = a.sq;
        d.tq = a.tq;
        d.out_off = out_off[v];
        d.ntx = (a.Wv + kWarpTW - 1) / kWarpTW;
        d.tile_start = per_view ? 0 : tiles;
        tiles += d.ntx * ((a.Hv + kWarpTH - 1) / kWarpTH);
        d.t = a.t;
        // exact trig at multiples of 90 degrees, as in the view table
        d.cosd = (double)a.cq / 2147483648.0;
        d.sind = (double)a.sq / 2147483648.0;
        {
            const double r = a.phi_deg * (3.14159265358979323846 / 180.0);
            if (std::fmod(a.phi_deg, 90.0) != 0.0) {
                d.cosd = std::cos(r);
                d.sind = std::sin(r);
            }
        }
        for (int k = 0; k < ASIFT_MAX_GAUSS; ++k) d.g[k] = (k <= a.K) ? a.g[k] : 0.f;
        int cw, bw;
        warp_strip_widths(a, &cw, &bw);
        cwm = std::max(cwm, cw);
        bwm = std::max(bwm, bw);
    }
    *n_tiles = tiles;
    *cw_max = cwm;
    *bw_max = bwm;
}

static bool view_ok(const asift_view_desc &v)
{
    return v.W >= 1 && v.H >= 1 && v.Wr >= 1 && v.Hr >= 1 && v.Wv >= 1 && v.Hv >= 1 && v.K >= 0 &&
           v.K < ASIFT_MAX_GAUSS && v.Wv < 32768 && v.Hv < 32768 && v.t >= 1.0;
}

}  // namespace asift

using namespace asift;

// ---------------------------------------------------------------- context
struct asift_ctx {
    int device = 0;
    asift_orb_cfg cfg{};
    int8_t h_pat[kBins][kPairs][4];
    long long h_bins[kBins][2];
    int *d_pat = nullptr;
    long long *d_bins = nullptr;
    static constexpr int kRing = 8;
    unsigned char *h_ring[kRing] = {};
    cudaEvent_t ring_ev[kRing] = {};
    size_t ring_cap = 0;
    int ring_next = 0;
    bool prof = false;
    cudaEvent_t prof_ev[ASIFT_PROF_STAGES + 1] = {};
};

static void prof_mark(asift_ctx *ctx, int i, cudaStream_t s)
{
    if (ctx->prof) cudaEventRecord(ctx->prof_ev[i], s);
}

static asift_status cuda_status(cudaError_t e) { return e == cudaSuccess ? ASIFT_OK : ASIFT_ERR_CUDA; }

// Copies n host bytes to device memory on `s` through the context's pinned
// ring (a slot is reused only after its previous copy has completed).
static cudaError_t upload(asift_ctx *ctx, void *dst, const void *src, size_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (n > ctx->ring_cap) return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);
    const int slot = ctx->ring_next;
    ctx->ring_next = (ctx->ring_next + 1) % asift_ctx::kRing;
    cudaError_t e = cudaEventSynchronize(ctx->ring_ev[slot]);
    if (e != cudaSuccess) return e;
    std::memcpy(ctx->h_ring[slot], src, n);
    e = cudaMemcpyAsync(dst, ctx->h_ring[slot], n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(ctx->ring_ev[slot], s);
}

extern "C" {

asift_status asift_ctx_create(asift_ctx **out, const asift_orb_cfg *cfg, uint64_t pattern_seed)
{
    if (!out) return ASIFT_ERR_ARG;
    *out = nullptr;
    asift_orb_cfg c{4, 500, 20, 60000};
    if (cfg) c = *cfg;
    if (c.n_levels < 1 || c.n_levels > ASIFT_MAX_LEVELS || c.n_features < 1 || c.n_features > 4096 ||
        c.fast_threshold < 0 || c.fast_threshold > 255 || c.cand_per_mpx < 0 || c.cand_per_mpx > 1000000)
        return ASIFT_ERR_ARG;
    asift_ctx *ctx = new (std::nothrow) asift_ctx;
    if (!ctx) return ASIFT_ERR_NOMEM;
    ctx->cfg = c;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) { delete ctx; return ASIFT_ERR_CUDA; }
    make_pattern(pattern_seed, ctx->h_pat);
    make_bin_table(ctx->h_bins);
    if (cudaMalloc(&ctx->d_pat, sizeof(ctx->h_pat)) != cudaSuccess ||
        cudaMalloc(&ctx->d_bins, sizeof(ctx->h_bins)) != cudaSuccess) {
        asift_ctx_destroy(ctx);
        return ASIFT_ERR_NOMEM;
    }
    if (cudaMemcpy(ctx->d_pat, ctx->h_pat, sizeof(ctx->h_pat), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_bins, ctx->h_bins, sizeof(ctx->h_bins), cudaMemcpyHostToDevice) != cudaSuccess) {
        asift_ctx_destroy(ctx);
        return ASIFT_ERR_CUDA;
    }
    ctx->ring_cap = 1 << 20;
    for (int i = 0; i < asift_ctx::kRing; ++i) {
        if (cudaHostAlloc(&ctx->h_ring[i], ctx->ring_cap, cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ring_ev[i], cudaEventDisableTiming) != cudaSuccess) {
            asift_ctx_destroy(ctx);
            return ASIFT_ERR_NOMEM;
        }
    }
    *out = ctx;
    return ASIFT_OK;
}

void asift_ctx_destroy(asift_ctx *ctx)
{
    if (!ctx) return;
    for (int i = 0; i < asift_ctx::kRing; ++i) {
        if (ctx->ring_ev[i]) {
            cudaEventSynchronize(ctx->ring_ev[i]);
            cudaEventDestroy(ctx->ring_ev[i]);
        }
        if (ctx->h_ring[i]) cudaFreeHost(ctx->h_ring[i]);
    }
    for (int i = 0; i <= ASIFT_PROF_STAGES; ++i)
        if (ctx->prof_ev[i]) cudaEventDestroy(ctx->prof_ev[i]);
    if (ctx->d_pat) cudaFree(ctx->d_pat);
    if (ctx->d_bins) cudaFree(ctx->d_bins);
    delete ctx;
}

asift_status asift_ctx_orb_cfg(const asift_ctx *ctx, asift_orb_cfg *out)
{
    if (!ctx || !out) return ASIFT_ERR_ARG;
    *out = ctx->cfg;
    return ASIFT_OK;
}

asift_status asift_ctx_pattern(const asift_ctx *ctx, int8_t *h_out)
{
    if (!ctx || !h_out) return ASIFT_ERR_ARG;
    std::memcpy(h_out, ctx->h_pat, sizeof(ctx->h_pat));
    return ASIFT_OK;
}

asift_status asift_view_table(int H, int W, int kmax, asift_view_desc *h_out, int cap, int *n_views)
{
    if (H < 1 || W < 1 || H > 16384 || W > 16384 || kmax < 0 || kmax > 7 || !n_views || cap < 0)
        return ASIFT_ERR_ARG;
    *n_views = view_table(H, W, kmax, h_out, cap);
    return ASIFT_OK;
}

asift_status asift_make_view(int H, int W, double t, double phi_deg, asift_view_desc *h_out)
{
    if (H < 1 || W < 1 || H > 16384 || W > 16384 || !(t >= 1.0 && t < 11.4) || !h_out || !(phi_deg == phi_deg))
        return ASIFT_ERR_ARG;
    make_view_desc(H, W, t, phi_deg, -1, -1, h_out);
    return ASIFT_OK;
}

int asift_level_size(int n0, int level) { return level_size(n0, level); }

asift_status asift_pattern_table(uint64_t seed, int8_t *h_out)
{
    if (!h_out) return ASIFT_ERR_ARG;
    make_pattern(seed, reinterpret_cast<int8_t(*)[256][4]>(h_out));
    return ASIFT_OK;
}

asift_status asift_bin_table(int64_t *h_out)
{
    if (!h_out) return ASIFT_ERR_ARG;
    make_bin_table(reinterpret_cast<long long(*)[2]>(h_out));
    return ASIFT_OK;
}

int64_t asift_views_bytes(const asift_view_desc *h_views, int n_views)
{
    int64_t s = 0;
    for (int i = 0; i < n_views; ++i) s += (int64_t)h_views[i].Wv * h_views[i].Hv;
    return s;
}

int64_t asift_launch_count(void) { return g_launches.load(); }

asift_status asift_profile_enable(asift_ctx *ctx, int on)
{
    if (!ctx) return ASIFT_ERR_ARG;
    if (on && !ctx->prof) {
        for (int i = 0; i <= ASIFT_PROF_STAGES; ++i)
            if (!ctx->prof_ev[i] && cudaEventCreate(&ctx->prof_ev[i]) != cudaSuccess) return ASIFT_ERR_CUDA;
    }
    ctx->prof = on != 0;
    return ASIFT_OK;
}

asift_status asift_profile_read(asift_ctx *ctx, float *h_ms, int n)
{
    if (!ctx || !h_ms || n < 0 || !ctx->prof) return ASIFT_ERR_ARG;
    if (cudaEventSynchronize(ctx->prof_ev[ASIFT_PROF_STAGES]) != cudaSuccess) return ASIFT_ERR_CUDA;
    for (int i = 0; i < n && i < ASIFT_PROF_STAGES; ++i)
        if (cudaEventElapsedTime(&h_ms[i], ctx->prof_ev[i], ctx->prof_ev[i + 1]) != cudaSuccess) return ASIFT_ERR_CUDA;
    return ASIFT_OK;
}

asift_status asift_read_status(void *d_workspace, int clear, int32_t *h_status, void *stream)
{
    if (!d_workspace || !h_status) return ASIFT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(h_status, d_workspace, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && clear) e = cudaMemsetAsync(d_workspace, 0, sizeof(int32_t), s);
    if (e == cudaSuccess && clear) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

// ---------------------------------------------------------------- asift_views
static size_t views_layout(void *base, int H, int W, int nv, int32_t **status, DevView **tab, float **src)
{
    Bump b(base);
    *status = b.take<int32_t>(64);
    *tab = b.take<DevView>(std::max(nv, 1));
    *src = b.take<float>((size_t)W * H);
    return b.off + 256;
}

size_t asift_views_workspace_size(int H, int W, int n_views)
{
    int32_t *s;
    DevView *t;
    float *f;
    return views_layout(nullptr, H, W, n_views, &s, &t, &f);
}

asift_status asift_views(asift_ctx *ctx, const uint8_t *d_img, int H, int W, int pitch,
                         const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                         float *d_view_f32, uint8_t *d_view_u8, uint8_t *d_mask, void *d_workspace,
                         size_t ws_bytes, void *stream)
{
    if (!ctx || !d_img || H < 1 || W < 1 || pitch < W || n_views < 0 || (n_views && (!h_views || !h_offsets)) ||
        !d_view_u8 || !d_mask || !d_workspace)
        return ASIFT_ERR_ARG;
    if (ws_bytes < asift_views_workspace_size(H, W, n_views)) return ASIFT_ERR_ARG;
    for (int v = 0; v < n_views; ++v)
        if (!view_ok(h_views[v]) || h_views[v].W != W || h_views[v].H != H || h_offsets[v] < 0) return ASIFT_ERR_ARG;
    if (n_views == 0) return ASIFT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *status;
    DevView *tab;
    float *src;
    views_layout(d_workspace, H, W, n_views, &status, &tab, &src);
    std::vector<const float *> srcs(n_views, src);
    std::vector<int> pitches(n_views, W);
    std::vector<DevView> dv;
    int n_tiles, cwm, bwm;
    build_views(h_views, n_views, srcs.data(), pitches.data(), h_offsets, false, dv, &n_tiles, &cwm, &bwm);
    cudaError_t e = upload(ctx, tab, dv.data(), sizeof(DevView) * n_views, s);
    if (e == cudaSuccess) e = launch_u8_to_f32(d_img, pitch, W, H, src, s);
    if (e == cudaSuccess) e = launch_warp(tab, n_views, n_tiles, cwm, bwm, d_view_u8, d_mask, d_view_f32, s);
    return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------- ORB pipeline
namespace asift {

struct OrbBuffers {
    int32_t *status;
    DevLevel *lv;
    int32_t *group_first;
    uint8_t *arena_u8, *arena_mask;
    int32_t *cand_count;
    Candidate *cand;
    SlotKp *slots;
    int32_t *taken, *pool_off;
    int32_t *group_total;
};

// Workspace region of the ORB stages for nv views in n_groups groups.
static void orb_layout(Bump &b, const LevelTables &T, int nv, int n_groups, const asift_orb_cfg &cfg, OrbBuffers &o)
{
    const size_t nl = (size_t)cfg.n_levels * nv;
    o.lv = b.take<DevLevel>(std::max<size_t>(nl, 1));
    o.group_first = b.take<int32_t>(n_groups + 1);
    o.arena_u8 = b.take<uint8_t>((size_t)T.arena_bytes + 16);
    o.arena_mask = b.take<uint8_t>((size_t)T.arena_bytes + 16);
    o.cand_count = b.take<int32_t>(nl);
    o.cand = b.take<Candidate>((size_t)T.cand_total);
    o.slots = b.take<SlotKp>((size_t)nv * cfg.n_features);
    o.taken = b.take<int32_t>(nl);
    o.pool_off = b.take<int32_t>(nl);
    o.group_total = b.take<int32_t>(n_groups);
}

// Runs pyramid -> detect -> select -> pool scan -> orientation + BRIEF.
// The level table and group boundaries must already be uploaded.
static cudaError_t run_orb(asift_ctx *ctx, const LevelTables &T, int nv, int n_groups, const OrbBuffers &o,
                           bool per_view, asift_keypoint *kp, uint8_t *desc, int32_t *view_count, int32_t *view_off,
                           cudaStream_t s)
{
    const asift_orb_cfg &cfg = ctx->cfg;
    const int L = cfg.n_levels, N = cfg.n_features;
    const size_t nl = (size_t)L * nv;
    cudaError_t e = cudaMemsetAsync(o.cand_count, 0, sizeof(int32_t) * nl, s);
    if (e != cudaSuccess) return e;
    if (!per_view) {
        for (int l = 1; l < L && e == cudaSuccess; ++l)
            e = launch_pyramid(o.lv + (size_t)l * nv, nv, T.pyr_tiles[l], s);
        prof_mark(ctx, 3, s);
        if (e == cudaSuccess)
            e = launch_detect(o.lv, (int)nl, T.det_tiles, cfg.fast_threshold, o.cand, o.cand_count, s);
        prof_mark(ctx, 4, s);
        if (e == cudaSuccess)
            e = launch_select(o.lv, (int)nl, o.cand, o.cand_count, N, o.slots, o.taken, o.status, s);
        prof_mark(ctx, 5, s);
    } else {
        prof_mark(ctx, 3, s);
        prof_mark(ctx, 4, s);
        for (int v = 0; v < nv && e == cudaSuccess; ++v) {
            for (int l = 1; l < L && e == cudaSuccess; ++l) {
                const size_t i = (size_t)l * nv + v;
                e = launch_pyramid(o.lv + i, 1, pyr_tiles_of(T.lv[i]), s);
            }
            for (int l = 0; l < L && e == cudaSuccess; ++l) {
                const size_t i = (size_t)l * nv + v;
                e = launch_detect(o.lv + i, 1, det_tiles_of(T.lv[i]), cfg.fast_threshold, o.cand, o.cand_count + i, s);
            }
            for (int l = 0; l < L && e == cudaSuccess; ++l) {
                const size_t i = (size_t)l * nv + v;
                e = launch_select(o.lv + i, 1, o.cand, o.cand_count + i, N, o.slots, o.taken + i, o.status, s);
            }
        }
        prof_mark(ctx, 5, s);
    }
    if (e == cudaSuccess)
        e = launch_pool_scan(o.taken, nv, L, o.group_first, n_groups, N, o.pool_off, view_count, view_off,
                             o.group_total, s);
    if (!per_view) {
        if (e == cudaSuccess)
            e = launch_orient_brief(o.lv, nv, L, N, 0, nv, o.slots, o.taken, o.pool_off, ctx->d_pat, ctx->d_bins, kp,
                                    reinterpret_cast<uint4 *>(desc), s);
    } else {
        for (int v = 0; v < nv && e == cudaSuccess; ++v)
            e = launch_orient_brief(o.lv, nv, L, N, v, v + 1, o.slots, o.taken, o.pool_off, ctx->d_pat, ctx->d_bins,
                                    kp, reinterpret_cast<uint4 *>(desc), s);
    }
    prof_mark(ctx, 6, s);
    return e;
}

}  // namespace asift

extern "C" {

static size_t orb_ws(const asift_ctx *ctx, const asift_view_desc *h_views, int n_views, void *base,
                     LevelTables *T_out, OrbBuffers *o_out, int32_t **vc, int32_t **vo)
{
    LevelTables T;
    std::vector<const uint8_t *> dummy(std::max(n_views, 1), nullptr);
    Bump b(base);
    int32_t *status = b.take<int32_t>(64);
    // first pass sizes the arena; pointers are filled in by the caller with the real base
    build_levels(ctx->cfg, h_views, n_views, dummy.data(), dummy.data(), nullptr, nullptr, false, T);
    OrbBuffers o;
    orb_layout(b, T, n_views, 1, ctx->cfg, o);
    o.status = status;
    int32_t *view_count = b.take<int32_t>(std::max(n_views, 1));
    int32_t *view_off = b.take<int32_t>(std::max(n_views, 1));
    if (T_out) *T_out = T;
    if (o_out) *o_out = o;
    if (vc) *vc = view_count;
    if (vo) *vo = view_off;
    return b.off + 256;
}

size_t orb_workspace_size(const asift_ctx *ctx, const asift_view_desc *h_views, int n_views)
{
    if (!ctx || n_views < 0 || (n_views && !h_views)) return 0;
    return orb_ws(ctx, h_views, n_views, nullptr, nullptr, nullptr, nullptr, nullptr);
}

asift_status orb_extract(asift_ctx *ctx, const uint8_t *d_view_u8, const uint8_t *d_mask,
                         const asift_view_desc *h_views, int n_views, const int64_t *h_offsets, asift_keypoint *d_kp,
                         uint8_t *d_desc, int32_t *d_view_count, int32_t *d_view_offset, int32_t *d_total,
                         void *d_workspace, size_t ws_bytes, void *stream)
{
    if (!ctx || !d_view_u8 || !d_mask || n_views < 1 || n_views > 65535 || !h_views || !h_offsets || !d_kp ||
        !d_desc || !d_view_count || !d_view_offset || !d_total || !d_workspace)
        return ASIFT_ERR_ARG;
    for (int v = 0; v < n_views; ++v)
        if (!view_ok(h_views[v]) || h_offsets[v] < 0) return ASIFT_ERR_ARG;
    if (ws_bytes < orb_workspace_size(ctx, h_views, n_views)) return ASIFT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LevelTables T;
    OrbBuffers o;
    int32_t *vc_ws, *vo_ws;
    orb_ws(ctx, h_views, n_views, d_workspace, &T, &o, &vc_ws, &vo_ws);
    std::vector<const uint8_t *> l0i(n_views), l0m(n_views);
    for (int v = 0; v < n_views; ++v) {
        l0i[v] = d_view_u8 + h_offsets[v];
        l0m[v] = d_mask + h_offsets[v];
    }
    build_levels(ctx->cfg, h_views, n_views, l0i.data(), l0m.data(), o.arena_u8, o.arena_mask, false, T);
    // level table and group boundaries in one upload (they are adjacent in the workspace)
    const size_t lv_bytes = sizeof(DevLevel) * T.lv.size();
    const size_t gap = (size_t)((char *)o.group_first - (char *)o.lv);
    std::vector<unsigned char> blob(gap + 2 * sizeof(int32_t));
    std::memcpy(blob.data(), T.lv.data(), lv_bytes);
    const int32_t gf[2] = {0, n_views};
    std::memcpy(blob.data() + gap, gf, sizeof(gf));
    cudaError_t e = upload(ctx, o.lv, blob.data(), blob.size(), s);
    if (e == cudaSuccess)
        e = run_orb(ctx, T, n_views, 1, o, false, d_kp, d_desc, d_view_count, d_view_offset, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_total, o.group_total, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    return cuda_status(e);
}

// ---------------------------------------------------------------- hamming_match
size_t hamming_workspace_size(int nq, int nt)
{
    Bump b(nullptr);
    b.take<int32_t>(64);
    b.take<unsigned char>(hamming_partial_bytes(std::max(nq, 1), std::max(nt, 0)));
    return b.off + 256;
}

asift_status hamming_match(asift_ctx *ctx, const uint8_t *d_q, int nq, const int32_t *d_nq, const uint8_t *d_t,
                           int nt, const int32_t *d_nt, int ratio_num, int ratio_den, asift_match *d_out,
                           uint8_t *d_accept, int32_t *d_n_accepted, void *d_workspace, size_t ws_bytes,
                           void *stream)
{
    if (!ctx || nq < 0 || nt < 0 || nt > (1 << 23) - 1 || (nq && (!d_q || !d_out)) || (nt && !d_t) ||
        ratio_num < 0 || ratio_den < 1 || ratio_num > (1 << 20) || ratio_den > (1 << 20) || !d_workspace)
        return ASIFT_ERR_ARG;
    if (ws_bytes < hamming_workspace_size(nq, nt)) return ASIFT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (d_n_accepted) e = cudaMemsetAsync(d_n_accepted, 0, sizeof(int32_t), s);
    if (nq == 0 || e != cudaSuccess) return cuda_status(e);
    Bump b(d_workspace);
    b.take<int32_t>(64);
    void *part = b.take<unsigned char>(hamming_partial_bytes(nq, nt));
    e = launch_hamming(d_q, nq, d_nq, d_t, nt, d_nt, ratio_num, ratio_den, d_out, d_accept, d_n_accepted, part, s);
    return cuda_status(e);
}

asift_status hamming_match_noalloc(const uint8_t *d_q, int nq, const int32_t *d_nq, const uint8_t *d_t, int nt,
                                   const int32_t *d_nt, int ratio_num, int ratio_den, asift_match *d_out,
                                   uint8_t *d_accept, int32_t *d_n_accepted, void *stream)
{
    if (nq < 0 || nt < 0 || nq > ASIFT_NOALLOC_MAX_QUERIES || nt > (1 << 23) - 1 || (nq && (!d_q || !d_out)) ||
        (nt && !d_t) || ratio_num < 0 || ratio_den < 1 || ratio_num > (1 << 20) || ratio_den > (1 << 20))
        return ASIFT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (d_n_accepted) e = cudaMemsetAsync(d_n_accepted, 0, sizeof(int32_t), s);
    if (nq == 0 || e != cudaSuccess) return cuda_status(e);
    e = launch_hamming_noalloc(d_q, nq, d_nq, d_t, nt, d_nt, ratio_num, ratio_den, d_out, d_accept, d_n_accepted, s);
    return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------- match_pair
namespace asift {

struct PairLayout {
    int nv1 = 0, nv2 = 0;
    std::vector<asift_view_desc> views;     // image 1 views then image 2 views
    std::vector<int64_t> level0_off;        // per view: offset of level 0 in the arena
    LevelTables T;
    int32_t *status = nullptr;
    DevView *dv = nullptr;
    OrbBuffers o{};
    float *src1 = nullptr, *src2 = nullptr;
    int32_t *view_count = nullptr, *view_off = nullptr;
    asift_keypoint *kp = nullptr;
    uint8_t *desc = nullptr;
    asift_match *match = nullptr;
    uint8_t *accept = nullptr;
    int32_t *n_acc = nullptr;
    void *part = nullptr;
    int32_t *block_count = nullptr;
    size_t bytes = 0;
};

static bool pair_layout(const asift_ctx *ctx, int H1, int W1, int H2, int W2, const asift_pair_cfg &pc, void *base,
                        bool per_view, PairLayout &P)
{
    const asift_orb_cfg &cfg = ctx->cfg;
    int n1 = view_table(H1, W1, pc.kmax, nullptr, 0), n2 = view_table(H2, W2, pc.kmax, nullptr, 0);
    P.nv1 = n1;
    P.nv2 = n2;
    P.views.resize(n1 + n2);
    view_table(H1, W1, pc.kmax, P.views.data(), n1);
    view_table(H2, W2, pc.kmax, P.views.data() + n1, n2);
    const int nv = n1 + n2;
    if (nv > 65535) return false;
    // level 0 of every view lives in the same arena as the other levels
    Bump b(base);
    P.status = b.take<int32_t>(64);
    P.dv = b.take<DevView>(nv);
    build_levels(cfg, P.views.data(), nv, nullptr, nullptr, nullptr, nullptr, per_view, P.T);
    orb_layout(b, P.T, nv, 2, cfg, P.o);
    P.o.status = P.status;
    // pointers of the level table with the real arena base
    build_levels(cfg, P.views.data(), nv, nullptr, nullptr, P.o.arena_u8, P.o.arena_mask, per_view, P.T);
    P.level0_off.resize(nv);
    for (int v = 0; v < nv; ++v)
        P.level0_off[v] = P.o.arena_u8 ? (int64_t)(P.T.lv[v].img - P.o.arena_u8) : 0;
    if (!base) {
        // offsets are needed for the table layout even in the size query
        long long off = 0;
        for (int v = 0; v < nv; ++v) {
            P.level0_off[v] = off;
            for (int l = 0; l < cfg.n_levels; ++l)
                off += ((long long)level_size(P.views[v].Wv, l) * level_size(P.views[v].Hv, l) + 15) & ~15LL;
        }
    }
    P.src1 = b.take<float>((size_t)W1 * H1);
    P.src2 = b.take<float>((size_t)W2 * H2);
    P.view_count = b.take<int32_t>(nv);
    P.view_off = b.take<int32_t>(nv);
    const size_t cap = (size_t)nv * cfg.n_features;
    P.kp = b.take<asift_keypoint>(cap);
    P.desc = b.take<uint8_t>(cap * 32);
    const int nq = n1 * cfg.n_features, nt = n2 * cfg.n_features;
    P.match = b.take<asift_match>(nq);
    P.accept = b.take<uint8_t>(nq);
    P.n_acc = b.take<int32_t>(1);
    P.part = b.take<unsigned char>(hamming_partial_bytes(nq, nt));
    P.block_count = b.take<int32_t>(pair_blocks(nq));
    P.bytes = b.off + 256;
    return true;
}

}  // namespace asift

extern "C" {

static asift_pair_cfg pair_cfg_or_default(const asift_pair_cfg *c)
{
    asift_pair_cfg d{5, 4, 5, 0};
    return c ? *c : d;
}

size_t match_pair_workspace_size(const asift_ctx *ctx, int H1, int W1, int H2, int W2, const asift_pair_cfg *cfg)
{
    if (!ctx || H1 < 1 || W1 < 1 || H2 < 1 || W2 < 1) return 0;
    const asift_pair_cfg pc = pair_cfg_or_default(cfg);
    if (pc.kmax < 0 || pc.kmax > 7) return 0;
    PairLayout P;
    if (!pair_layout(ctx, H1, W1, H2, W2, pc, nullptr, pc.per_view != 0, P)) return 0;
    return P.bytes;
}

asift_status match_pair(asift_ctx *ctx, const uint8_t *d_img1, int H1, int W1, int pitch1, const uint8_t *d_img2,
                        int H2, int W2, int pitch2, const asift_pair_cfg *cfg, asift_pair_match *d_out, int cap,
                        int32_t *d_n, void *d_workspace, size_t ws_bytes, void *stream)
{
    const asift_pair_cfg pc = pair_cfg_or_default(cfg);
    if (!ctx || !d_img1 || !d_img2 || H1 < 1 || W1 < 1 || H2 < 1 || W2 < 1 || H1 > 16384 || W1 > 16384 ||
        H2 > 16384 || W2 > 16384 || pitch1 < W1 || pitch2 < W2 || pc.kmax < 0 || pc.kmax > 7 || pc.ratio_den < 1 ||
        pc.ratio_num < 0 || cap < 0 || (cap && !d_out) || !d_n || !d_workspace)
        return ASIFT_ERR_ARG;
    const bool per_view = pc.per_view != 0;
    PairLayout P;
    if (!pair_layout(ctx, H1, W1, H2, W2, pc, d_workspace, per_view, P)) return ASIFT_ERR_ARG;
    if (ws_bytes < P.bytes) return ASIFT_ERR_ARG;
    const asift_orb_cfg &oc = ctx->cfg;
    const int nv = P.nv1 + P.nv2, N = oc.n_features;
    const int nq = P.nv1 * N, nt = P.nv2 * N;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // host tables: views (warp) + levels (ORB) + group boundaries, one upload
    std::vector<const float *> srcs(nv);
    std::vector<int> pitches(nv);
    for (int v = 0; v < nv; ++v) {
        srcs[v] = v < P.nv1 ? P.src1 : P.src2;
        pitches[v] = v < P.nv1 ? W1 : W2;
    }
    std::vector<DevView> dv;
    int n_tiles, cwm, bwm;
    build_views(P.views.data(), nv, srcs.data(), pitches.data(), P.level0_off.data(), per_view, dv, &n_tiles, &cwm,
                &bwm);
    const size_t tab_end = (size_t)((char *)P.o.group_first - (char *)P.dv) + 3 * sizeof(int32_t);
    std::vector<unsigned char> blob(tab_end);
    std::memcpy(blob.data(), dv.data(), sizeof(DevView) * nv);
    std::memcpy(blob.data() + ((char *)P.o.lv - (char *)P.dv), P.T.lv.data(), sizeof(DevLevel) * P.T.lv.size());
    const int32_t gf[3] = {0, P.nv1, nv};
    std::memcpy(blob.data() + ((char *)P.o.group_first - (char *)P.dv), gf, sizeof(gf));

    prof_mark(ctx, 0, s);
    cudaError_t e = upload(ctx, P.dv, blob.data(), blob.size(), s);
    if (e == cudaSuccess) e = launch_u8_to_f32(d_img1, pitch1, W1, H1, P.src1, s);
    if (e == cudaSuccess) e = launch_u8_to_f32(d_img2, pitch2, W2, H2, P.src2, s);
    prof_mark(ctx, 1, s);
    if (e == cudaSuccess) {
        if (!per_view) {
            e = launch_warp(P.dv, nv, n_tiles, cwm, bwm, P.o.arena_u8, P.o.arena_mask, nullptr, s);
        } else {
            for (int v = 0; v < nv && e == cudaSuccess; ++v) {
                const int tiles = dv[v].ntx * ((P.views[v].Hv + kWarpTH - 1) / kWarpTH);
                e = launch_warp(P.dv + v, 1, tiles, cwm, bwm, P.o.arena_u8, P.o.arena_mask, nullptr, s);
            }
        }
    }
    prof_mark(ctx, 2, s);
    if (e == cudaSuccess) e = run_orb(ctx, P.T, nv, 2, P.o, per_view, P.kp, P.desc, P.view_count, P.view_off, s);
    // pool 1 = views of image 1 (slice 0), pool 2 = views of image 2 (slice nv1 * N)
    if (e == cudaSuccess)
        e = cudaMemsetAsync(P.n_acc, 0, sizeof(int32_t), s);
    if (e == cudaSuccess)
        e = launch_hamming(P.desc, nq, P.o.group_total, P.desc + (size_t)P.nv1 * N * 32, nt, P.o.group_total + 1,
                           pc.ratio_num, pc.ratio_den, P.match, P.accept, P.n_acc, P.part, s);
    prof_mark(ctx, 7, s);
    if (e == cudaSuccess)
        e = launch_pairs(P.accept, P.match, nq, P.o.group_total, P.block_count, P.kp, P.kp + (size_t)P.nv1 * N, P.dv,
                         d_out, cap, d_n, P.status, s);
    prof_mark(ctx, 8, s);
    return cuda_status(e);
}

asift_status match_pair_inspect(const asift_ctx *ctx, int H1, int W1, int H2, int W2, const asift_pair_cfg *cfg,
                                void *d_workspace, asift_keypoint **d_kp1, uint8_t **d_desc1, int32_t **d_n1,
                                asift_keypoint **d_kp2, uint8_t **d_desc2, int32_t **d_n2, asift_match **d_match)
{
    if (!ctx || !d_workspace) return ASIFT_ERR_ARG;
    const asift_pair_cfg pc = pair_cfg_or_default(cfg);
    PairLayout P;
    if (!pair_layout(ctx, H1, W1, H2, W2, pc, d_workspace, pc.per_view != 0, P)) return ASIFT_ERR_ARG;
    const size_t off2 = (size_t)P.nv1 * ctx->cfg.n_features;
    if (d_kp1) *d_kp1 = P.kp;
    if (d_desc1) *d_desc1 = P.desc;
    if (d_n1) *d_n1 = P.o.group_total;
    if (d_kp2) *d_kp2 = P.kp + off2;
    if (d_desc2) *d_desc2 = P.desc + off2 * 32;
    if (d_n2) *d_n2 = P.o.group_total + 1;
    if (d_match) *d_match = P.match;
    return ASIFT_OK;
}

}  // extern "C"
