// api.cu -- the C ABI of libasift (include/asift.h): contexts, workspace
// layouts, and the launch sequences of asift_views, orb_extract,
// hamming_match and match_pair.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace asift {

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Per-device, per-kernel memo of the dynamic shared-memory limit already set,
// so launches pay for cudaFuncSetAttribute only when a larger size is needed.
// (The opt-in matters below 48 KB of dynamic memory too: the 48 KB default
// covers static plus dynamic shared memory.)
cudaError_t ensure_dynamic_smem(const void *func, size_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(func, dev);
    const auto it = set.find(key);
    if (it != set.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) set[key] = bytes;
    return e;
}

// SM count of the current device (cached per device).
int device_sm_count()
{
    static std::atomic<int> cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 152;
    if (dev >= 0 && dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

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
    long long rows_total = 0;     // rows of all levels (mask row hulls)
    long long rows_level0 = 0;    // of which level 0 (the first entries)
};

// cap_override > 0 (a failure-path test hook) replaces the configured capacity.
static int cand_capacity(const asift_orb_cfg &cfg, int W, int H, int cap_override)
{
    const long long c = cap_override > 0 ? cap_override : 4096 + (long long)cfg.cand_per_mpx * W * H / 1000000;
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

// The back-projection of level l of view a: level pixel (x, y) -> view pixel
// x0 = (x + 1/2) Wv / Wl - 1/2, y0 likewise with Hv / Hl; canvas offset
// dx = t (x0 - (Wv - 1)/2), dy = y0 - (Hr - 1)/2; source point
// (cos dx + sin dy) / s + (W - 1)/2, (-sin dx + cos dy) / s + (H - 1)/2, with
// exact trig at multiples of 90 degrees as in the view table.  Composed into
// one affine map in fp64.
static void backprojection_map(const asift_view_desc &a, int l, double bp[6])
{
    double c = std::cos(a.phi_deg * (3.14159265358979323846 / 180.0));
    double sn = std::sin(a.phi_deg * (3.14159265358979323846 / 180.0));
    if (std::fmod(a.phi_deg, 90.0) == 0.0) {
        const long q = ((long)(a.phi_deg / 90.0) % 4 + 4) % 4;
        c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
        sn = (q == 1) ? 1.0 : (q == 3 ? -1.0 : 0.0);
    }
    const double cs = c / a.s, ss = sn / a.s;
    const double rx = (double)a.Wv / (double)level_size(a.Wv, l), ry = (double)a.Hv / (double)level_size(a.Hv, l);
    // dx = ax x + bx, dy = ay y + by
    const double ax = a.t * rx, bx = a.t * (0.5 * rx - 0.5 - (a.Wv - 1) * 0.5);
    const double ay = ry, by = 0.5 * ry - 0.5 - (a.Hr - 1) * 0.5;
    bp[0] = cs * ax;
    bp[1] = ss * ay;
    bp[2] = cs * bx + ss * by + (a.W - 1) * 0.5;
    bp[3] = -ss * ax;
    bp[4] = cs * ay;
    bp[5] = -ss * bx + cs * by + (a.H - 1) * 0.5;
}

// Level tables of n views.  Level 0 of view v is (l0_img[v], l0_mask[v]) when
// given, otherwise it lives in the arena like the other levels.  per_view:
// every tile_start is 0 (each entry is launched on its own).
static void build_levels(const asift_orb_cfg &cfg, const asift_view_desc *views, int nv,
                         const uint8_t *const *l0_img, const uint8_t *const *l0_mask, uint8_t *arena_u8,
                         uint8_t *arena_mask, bool per_view, LevelTables &T, int cand_cap_override = 0)
{
    const int L = cfg.n_levels;
    T.lv.assign((size_t)L * nv, DevLevel{});
    T.pyr_tiles.assign(L, 0);
    T.det_tiles = 0;
    T.cand_total = 0;
    T.arena_bytes = 0;
    T.rows_total = 0;
    T.rows_level0 = 0;
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
            d.cand_cap = cand_capacity(cfg, d.W, d.H, cand_cap_override);
            d.cand_off = (int)T.cand_total;
            T.cand_total += d.cand_cap;
            backprojection_map(views[v], l, d.bp);
            d.row_off = (int)T.rows_total;
            T.rows_total += d.H;
            if (l == 0) T.rows_level0 += d.H;
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
// Floats of the per-column Gaussian + tilt filters of a view list.
static size_t tilt_filter_floats(const asift_view_desc *h, int nv)
{
    size_t n = 0;
    for (int v = 0; v < nv; ++v) n += (size_t)h[v].Wv * tilt_filter_pitch(h[v].K);
    return n;
}

// H: device array of tilt_filter_floats(h, nv) floats (the views' filters,
// view after view).
static void build_views(const asift_view_desc *h, int nv, const float *const *src, const int *src_pitch,
                        const int64_t *out_off, bool per_view, float *H, std::vector<DevView> &out, int *n_tiles,
                        int *cw_max, int *hp_max, int *max_wv)
{
    out.assign(nv, DevView{});
    int tiles = 0, cwm = 1, hpm = 4, wvm = 0;
    size_t hoff = 0;
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
        d.tw = warp_tile_width(a);
        d.ntx = (a.Wv + d.tw - 1) / d.tw;
        {
            int lx = 32, pitch = 72;
            warp_lane_layout(a.cq, a.sq, &lx, &pitch);
            d.lanes_x = (int16_t)lx;
            d.stage_pitch = (int16_t)pitch;
        }
        d.tile_start = per_view ? 0 : tiles;
        tiles += d.ntx * ((a.Hv + kWarpTH - 1) / kWarpTH);
        for (int k = 0; k < ASIFT_MAX_GAUSS; ++k) d.g[k] = (k <= a.K) ? a.g[k] : 0.f;
        d.hp = tilt_filter_pitch(a.K);
        d.filt = H ? H + hoff : nullptr;
        hoff += (size_t)a.Wv * d.hp;
        int cw, bw;
        warp_strip_widths(a, d.tw, &cw, &bw);
        cwm = std::max(cwm, cw);
        hpm = std::max(hpm, d.hp);
        wvm = std::max(wvm, a.Wv);
    }
    *n_tiles = tiles;
    *cw_max = cwm;
    *hp_max = hpm;
    *max_wv = wvm;
}

static bool view_ok(const asift_view_desc &v)
{
    return v.W >= 1 && v.H >= 1 && v.Wr >= 1 && v.Hr >= 1 && v.Wv >= 1 && v.Hv >= 1 && v.K >= 0 &&
           v.K < ASIFT_MAX_GAUSS && v.Wv < 32768 && v.Hv < 32768 && v.t >= 1.0 && v.s >= 1.0 && v.s <= 8.0;
}

}  // namespace asift

using namespace asift;

// ---------------------------------------------------------------- context
namespace asift {
struct PairCache;                       // match_pair's host tables of recent calls (below)
static void pair_cache_free(PairCache *c);
}  // namespace asift

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
    int match_engine = ASIFT_MATCH_AUTO;
    PairCache *pair_cache = nullptr;
    // failure-path test hooks (asift_ctx_set_test_hook; 0 = off)
    int test_cand_cap = 0;
    unsigned long long test_stall_ns = 0;
};

// The matcher engine a call uses: the tuning's, else the context's; AUTO
// resolves to tensor cores when the device has them.
static int resolve_engine(const asift_ctx *ctx, const asift_tuning *tune)
{
    int e = (tune && tune->match_engine) ? tune->match_engine : ctx->match_engine;
    if (e == ASIFT_MATCH_AUTO) e = tc_match_available() ? ASIFT_MATCH_TENSOR_CORES : ASIFT_MATCH_CUDA_CORES;
    return e;
}

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
    pair_cache_free(ctx->pair_cache);
    delete ctx;
}

asift_status asift_ctx_set_match_engine(asift_ctx *ctx, int engine)
{
    if (!ctx || engine < ASIFT_MATCH_AUTO || engine > ASIFT_MATCH_TENSOR_CORES) return ASIFT_ERR_ARG;
    ctx->match_engine = engine;
    return ASIFT_OK;
}

int asift_ctx_match_engine(const asift_ctx *ctx) { return ctx ? resolve_engine(ctx, nullptr) : 0; }

asift_status asift_ctx_set_test_hook(asift_ctx *ctx, int hook, int64_t value)
{
    if (!ctx) return ASIFT_ERR_ARG;
    switch (hook) {
    case ASIFT_HOOK_CAND_CAP:
        if (value < 0 || value > (1 << 30)) return ASIFT_ERR_ARG;
        ctx->test_cand_cap = (int)value;
        break;
    case ASIFT_HOOK_MATCH_STALL:
        if (value != 0 && (value < 1000 || value > 4000000000LL)) return ASIFT_ERR_ARG;
        ctx->test_stall_ns = (unsigned long long)value;
        break;
    default:
        return ASIFT_ERR_ARG;
    }
    pair_cache_free(ctx->pair_cache);   // cached layouts carry the old capacities
    ctx->pair_cache = nullptr;
    return ASIFT_OK;
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
    make_view_desc(H, W, t, phi_deg, -1, -1, 1.0, h_out);
    return ASIFT_OK;
}

asift_status asift_view_table_scaled(int H, int W, int kmax, double ds, asift_view_desc *h_out, int cap,
                                     int *n_views)
{
    if (H < 1 || W < 1 || H > 16384 || W > 16384 || kmax < 0 || kmax > 7 || !n_views || cap < 0 ||
        !(ds >= 0.0 && ds <= 2.0))
        return ASIFT_ERR_ARG;
    *n_views = view_table_scaled(H, W, kmax, ds, h_out, cap);
    return ASIFT_OK;
}

asift_status asift_make_view_scaled(int H, int W, double t, double phi_deg, double s, asift_view_desc *h_out)
{
    if (H < 1 || W < 1 || H > 16384 || W > 16384 || !(t >= 1.0 && t < 11.4) || !h_out || !(phi_deg == phi_deg) ||
        !(s >= 1.0 && s <= 8.0))
        return ASIFT_ERR_ARG;
    make_view_desc(H, W, t, phi_deg, -1, -1, s, h_out);
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
static size_t views_layout(void *base, int H, int W, int nv, size_t n_filter, int32_t **status, DevView **tab,
                           DevRotGroup **grp, float **src, float **filt)
{
    Bump b(base);
    *status = b.take<int32_t>(64);
    *tab = b.take<DevView>(std::max(nv, 1));
    *grp = b.take<DevRotGroup>(std::max(nv, 1));
    *src = b.take<float>((size_t)src_pitch_of(W) * H);
    *filt = b.take<float>(std::max<size_t>(n_filter, 1));
    return b.off + 256;
}

size_t asift_views_workspace_size(int H, int W, int n_views)
{
    // filters: at most Wv * pitch(K) floats per view, bounded by the largest
    // view of the image (Wv <= (W + H) / t + 1, K <= ASIFT_MAX_GAUSS - 1)
    const size_t per_view = (size_t)(W + H + 2) * tilt_filter_pitch(ASIFT_MAX_GAUSS - 1);
    int32_t *s;
    DevView *t;
    DevRotGroup *r;
    float *f, *g;
    return views_layout(nullptr, H, W, n_views, per_view * std::max(n_views, 1), &s, &t, &r, &f, &g);
}

static asift_status views_impl(asift_ctx *ctx, const uint8_t *d_img, int H, int W, int pitch,
                               const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                               float *d_view_f32, uint8_t *d_view_u8, uint8_t *d_mask, void *d_workspace,
                               size_t ws_bytes, void *stream, int interp)
{
    if (!ctx || !d_img || H < 1 || W < 1 || pitch < W || n_views < 0 || (n_views && (!h_views || !h_offsets)) ||
        !d_view_u8 || !d_mask || !d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
        return ASIFT_ERR_ARG;
    if (ws_bytes < asift_views_workspace_size(H, W, n_views)) return ASIFT_ERR_ARG;
    for (int v = 0; v < n_views; ++v)
        if (!view_ok(h_views[v]) || h_views[v].W != W || h_views[v].H != H || h_offsets[v] < 0) return ASIFT_ERR_ARG;
    if (n_views == 0) return ASIFT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *status;
    DevView *tab;
    DevRotGroup *grp;
    float *src, *filt;
    views_layout(d_workspace, H, W, n_views, tilt_filter_floats(h_views, n_views), &status, &tab, &grp, &src, &filt);
    std::vector<const float *> srcs(n_views, src);
    std::vector<int> pitches(n_views, src_pitch_of(W));
    std::vector<DevView> dv;
    int n_tiles, cwm, hpm, wvm;
    build_views(h_views, n_views, srcs.data(), pitches.data(), h_offsets, false, filt, dv, &n_tiles, &cwm, &hpm, &wvm);
    cudaError_t e = upload(ctx, tab, dv.data(), sizeof(DevView) * n_views, s);
    if (e == cudaSuccess) e = launch_u8_to_f32(d_img, pitch, W, H, src, src_pitch_of(W), s);
    if (interp == ASIFT_INTERP_NEAREST) {
        if (e == cudaSuccess) e = launch_warp_nn(tab, n_views, n_tiles, cwm, d_view_u8, d_mask, d_view_f32, s);
        return cuda_status(e);
    }
    if (interp == 3 || interp == 4) {       // Lanczos-a, the precise stage's kernel
        int lzw = 1;
        for (int v = 0; v < n_views; ++v) lzw = std::max(lzw, warp_lz_strip_width(h_views[v], dv[v].tw, interp));
        if (e == cudaSuccess)
            e = launch_warp_lanczos(interp, tab, n_views, n_tiles, lzw, d_view_u8, d_mask, d_view_f32, s);
        return cuda_status(e);
    }
    std::vector<DevRotGroup> groups;
    int g_tiles = 0, hk_max = 3;
    const int seg_w = warp_seg_width_default();
    build_rot_groups(h_views, dv.data(), n_views, false, seg_w, groups, &g_tiles, &hk_max);
    if (e == cudaSuccess) e = upload(ctx, grp, groups.data(), sizeof(DevRotGroup) * groups.size(), s);
    if (e == cudaSuccess) e = launch_tilt_filter(tab, n_views, wvm, s);
    if (e == cudaSuccess)
        e = launch_warp(grp, (int)groups.size(), tab, g_tiles, seg_w, hk_max, d_view_u8, d_mask, d_view_f32, s);
    return cuda_status(e);
}

asift_status asift_views(asift_ctx *ctx, const uint8_t *d_img, int H, int W, int pitch,
                         const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                         float *d_view_f32, uint8_t *d_view_u8, uint8_t *d_mask, void *d_workspace,
                         size_t ws_bytes, void *stream)
{
    return views_impl(ctx, d_img, H, W, pitch, h_views, n_views, h_offsets, d_view_f32, d_view_u8, d_mask,
                      d_workspace, ws_bytes, stream, ASIFT_INTERP_LANCZOS3);
}

asift_status asift_views_nearest(asift_ctx *ctx, const uint8_t *d_img, int H, int W, int pitch,
                                 const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                                 float *d_view_f32, uint8_t *d_view_u8, uint8_t *d_mask, void *d_workspace,
                                 size_t ws_bytes, void *stream)
{
    return views_impl(ctx, d_img, H, W, pitch, h_views, n_views, h_offsets, d_view_f32, d_view_u8, d_mask,
                      d_workspace, ws_bytes, stream, ASIFT_INTERP_NEAREST);
}

asift_status asift_views_lanczos(asift_ctx *ctx, int a, const uint8_t *d_img, int H, int W, int pitch,
                                 const asift_view_desc *h_views, int n_views, const int64_t *h_offsets,
                                 float *d_view_f32, uint8_t *d_view_u8, uint8_t *d_mask, void *d_workspace,
                                 size_t ws_bytes, void *stream)
{
    if (a != 3 && a != 4) return ASIFT_ERR_ARG;
    return views_impl(ctx, d_img, H, W, pitch, h_views, n_views, h_offsets, d_view_f32, d_view_u8, d_mask,
                      d_workspace, ws_bytes, stream, a);
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
    int32_t *row_lo, *row_hi;    // mask row hulls of every level (row_off of each entry)
    int32_t *unit;               // per view: nonzero when its masks are exactly their row hulls
    DetItem *det_list;           // the detection tiles worth processing, and their count
    int32_t *det_count;
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
    o.row_lo = b.take<int32_t>(std::max<long long>(T.rows_total, 1));
    o.row_hi = b.take<int32_t>(std::max<long long>(T.rows_total, 1));
    o.unit = b.take<int32_t>(std::max(nv, 1));
    o.det_list = b.take<DetItem>(std::max<long long>(T.det_tiles, 1));
    o.det_count = b.take<int32_t>(1);
}

// Runs pyramid -> detect -> select -> pool scan -> orientation + BRIEF.
// The level table and group boundaries must already be uploaded.
static cudaError_t run_orb(asift_ctx *ctx, const LevelTables &T, int nv, int n_groups, const OrbBuffers &o,
                           bool per_view, asift_keypoint *kp, uint8_t *desc, int32_t *view_count, int32_t *view_off,
                           cudaStream_t s, const asift_tuning *tune = nullptr)
{
    // untuned calls run the pyramid on a persistent grid of four CTAs per SM
    // (0.272 -> 0.262 ms on a 1024x768 pair against one CTA per tile); a
    // tuned plan takes its own choice (0 there is one CTA per tile)
    const int pyr_grid = tune ? tune->pyramid_grid : 4 * device_sm_count();
    const int det_grid = tune ? tune->detect_grid : 0;
    const asift_orb_cfg &cfg = ctx->cfg;
    const int L = cfg.n_levels, N = cfg.n_features;
    const size_t nl = (size_t)L * nv;
    cudaError_t e = cudaMemsetAsync(o.cand_count, 0, sizeof(int32_t) * nl, s);
    if (e != cudaSuccess) return e;
    // mask row hulls: level 0 scanned, levels >= 1 derived through the pyramid's taps
    int max_h1 = 0;   // the tallest level >= 1 (one thread per row of each)
    for (size_t i = (size_t)nv; i < T.lv.size(); ++i) max_h1 = std::max(max_h1, T.lv[i].H);
    e = launch_mask_rows(o.lv, nv, L, (int)T.rows_level0, max_h1, o.row_lo, o.row_hi, o.unit, s);
    if (e != cudaSuccess) return e;
    if (!per_view) {
        for (int l = 1; l < L && e == cudaSuccess; ++l)
            e = launch_pyramid(o.lv + (size_t)l * nv, nv, T.pyr_tiles[l], o.unit, s, pyr_grid);
        prof_mark(ctx, 3, s);
        if (e == cudaSuccess)
            e = launch_detect(o.lv, (int)nl, T.det_tiles, cfg.fast_threshold, o.cand, o.cand_count, o.row_lo, o.row_hi,
                              o.unit, o.det_list, o.det_count, s, det_grid);
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
                e = launch_pyramid(o.lv + i, 1, pyr_tiles_of(T.lv[i]), o.unit, s);
            }
            for (int l = 0; l < L && e == cudaSuccess; ++l) {
                const size_t i = (size_t)l * nv + v;
                e = launch_detect(o.lv + i, 1, det_tiles_of(T.lv[i]), cfg.fast_threshold, o.cand, o.cand_count + i,
                                  o.row_lo, o.row_hi, o.unit, o.det_list, o.det_count, s);
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
    build_levels(ctx->cfg, h_views, n_views, dummy.data(), dummy.data(), nullptr, nullptr, false, T, ctx->test_cand_cap);
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
    build_levels(ctx->cfg, h_views, n_views, l0i.data(), l0m.data(), o.arena_u8, o.arena_mask, false, T,
                 ctx->test_cand_cap);
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
// Workspace: status word, partial keys, then the expanded (+-1 fp8) queries
// and trains of the tensor-core engine.
struct HammingWs {
    int32_t *status;
    void *part;
    uint8_t *xq, *xt;
};

static size_t hamming_ws(void *base, int nq, int nt, HammingWs *w)
{
    Bump b(base);
    int32_t *status = b.take<int32_t>(64);
    void *part = b.take<unsigned char>(hamming_partial_bytes(std::max(nq, 1), std::max(nt, 0)));
    uint8_t *xq = b.take<uint8_t>(tc_expanded_bytes(nq));
    uint8_t *xt = b.take<uint8_t>(tc_expanded_bytes(nt));
    if (w) *w = HammingWs{status, part, xq, xt};
    return b.off + 256;
}

size_t hamming_workspace_size(int nq, int nt) { return hamming_ws(nullptr, std::max(nq, 0), std::max(nt, 0), nullptr); }

asift_status hamming_match(asift_ctx *ctx, const uint8_t *d_q, int nq, const int32_t *d_nq, const uint8_t *d_t,
                           int nt, const int32_t *d_nt, int ratio_num, int ratio_den, asift_match *d_out,
                           uint8_t *d_accept, int32_t *d_n_accepted, void *d_workspace, size_t ws_bytes,
                           void *stream)
{
    if (!ctx || nq < 0 || nt < 0 || nt > (1 << 23) - 1 || (nq && (!d_q || !d_out)) || (nt && !d_t) ||
        ratio_num < 0 || ratio_den < 1 || ratio_num > (1 << 20) || ratio_den > (1 << 20) || !d_workspace)
        return ASIFT_ERR_ARG;
    if (ws_bytes < hamming_workspace_size(nq, nt) || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
        return ASIFT_ERR_ARG;
    const int engine = resolve_engine(ctx, nullptr);
    if (engine == ASIFT_MATCH_TENSOR_CORES && !tc_match_available()) return ASIFT_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HammingWs w;
    hamming_ws(d_workspace, nq, nt, &w);
    cudaError_t e = cudaMemsetAsync(w.status, 0, sizeof(int32_t), s);
    if (d_n_accepted && e == cudaSuccess) e = cudaMemsetAsync(d_n_accepted, 0, sizeof(int32_t), s);
    if (nq == 0 || e != cudaSuccess) return cuda_status(e);
    if (engine == ASIFT_MATCH_TENSOR_CORES && nt > 0) {
        MatchProblem P;
        match_problem_init(P, d_q, nq, d_nq, d_t, nt, d_nt, w.part, 0, d_out, d_accept, d_n_accepted);
        e = launch_expand(d_q, w.xq, nullptr, 0, d_nq, nq, 1, s);
        if (e == cudaSuccess) e = launch_expand(d_t, w.xt, nullptr, 0, d_nt, nt, 1, s);
        if (e == cudaSuccess)
            e = launch_match_tc(d_q, w.xq, nq, d_t, w.xt, nt, nullptr, 0, P, nq, ratio_num, ratio_den,
                                MatchTuning{0, 0, ctx->test_stall_ns}, w.status, s);
    } else {
        e = launch_hamming(d_q, nq, d_nq, d_t, nt, d_nt, ratio_num, ratio_den, d_out, d_accept, d_n_accepted, w.part,
                           s);
    }
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

// ---------------------------------------------------------------- pair pipeline
// The whole hot path for P image pairs at once: the views of all 2P images in
// one warp launch, ORB over all of them (one pool slice per image), and P
// matching problems in one matcher launch.  match_pair is the case P = 1; the
// plan API captures the same sequence in a CUDA graph.
namespace asift {

struct PairSpec {
    int H1, W1, H2, W2;
};

struct Pipeline {
    int n_pairs = 0;
    std::vector<int> nv1, nv2;               // views per image
    std::vector<int> first;                  // view index of each image's first view (2P + 1)
    std::vector<asift_view_desc> views;      // all views, image by image
    std::vector<int64_t> level0_off;         // per view: level-0 offset in the arena
    LevelTables T;
    int nv = 0;
    // device regions
    int32_t *status = nullptr;
    DevView *dv = nullptr;
    OrbBuffers o{};
    MatchProblem *probs = nullptr;
    ImageConv *conv = nullptr;
    DevRotGroup *grp = nullptr;              // rotation groups of the Lanczos-3 warp
    std::vector<float *> src;                // fp32 copy of each image
    int32_t *view_count = nullptr, *view_off = nullptr;
    asift_keypoint *kp = nullptr;
    uint8_t *desc = nullptr;
    uint8_t *xdesc = nullptr;                // desc expanded to +-1 fp8 (tensor-core matcher)
    asift_match *match = nullptr;
    uint8_t *accept = nullptr;
    int32_t *n_acc = nullptr;
    std::vector<void *> part;                // matcher partials per problem
    int32_t *block_count = nullptr;
    // host copies of the device tables (uploaded as one blob from dv)
    std::vector<DevView> h_dv;
    std::vector<MatchProblem> h_probs;
    std::vector<ImageConv> h_conv;
    std::vector<DevRotGroup> h_grp;
    int grp_tiles = 0, hk_max = 3, seg_w = 0;
    int n_tiles = 0, cw_max = 0, hp_max = 0, max_wv = 0, total_q = 0, total_blk = 0, n_per_view = 0;
    float *tilt_filters = nullptr;           // per view column: Gaussian + tilt filter
    long long cap_rows = 0;
    long long max_px = 0;
    size_t tab_bytes = 0;                    // bytes from dv to the end of the table region
    size_t bytes = 0;
};

// match_pair's layout and host tables are a function of its arguments and of
// the context's (fixed) ORB configuration.  The context keeps those of its
// last few distinct calls, so a call that repeats one (a caller streaming
// pairs through the same buffers) goes straight to the upload and launches.
struct PairKey {
    const uint8_t *img1, *img2;
    int H1, W1, pitch1, H2, W2, pitch2;
    int32_t kmax, ratio_num, ratio_den, per_view, coarse, interp;
    double ds;
    asift_pair_match *out;
    int cap;
    int32_t *d_n;
    void *ws;
    bool operator==(const PairKey &o) const
    {
        return img1 == o.img1 && img2 == o.img2 && H1 == o.H1 && W1 == o.W1 && pitch1 == o.pitch1 && H2 == o.H2 &&
               W2 == o.W2 && pitch2 == o.pitch2 && kmax == o.kmax && ratio_num == o.ratio_num &&
               ratio_den == o.ratio_den && per_view == o.per_view && coarse == o.coarse && interp == o.interp && ds == o.ds &&
               out == o.out &&
               cap == o.cap && d_n == o.d_n && ws == o.ws;
    }
};

struct PairCache {
    static constexpr size_t kEntries = 4;
    struct Entry {
        PairKey key;
        Pipeline L;
        std::vector<unsigned char> blob;
        unsigned long long used = 0;
    };
    std::vector<Entry> e;
    unsigned long long clock = 0;
};

static void pair_cache_free(PairCache *c) { delete c; }

// The views of one pair: both images the sampling rule's (kmax), or for the
// coarse stage image 1 the scaled parameter groups (kmax, ds) and image 2 its
// single unwarped view.
static int pair_views(const PairSpec &p, const asift_pair_cfg &pc, int image, asift_view_desc *out, int cap)
{
    const int H = image ? p.H2 : p.H1, W = image ? p.W2 : p.W1;
    if (!pc.coarse) return view_table(H, W, pc.kmax, out, cap);
    return image ? view_table(H, W, 0, out, cap) : view_table_scaled(H, W, pc.kmax, pc.ds, out, cap);
}

static bool pair_cfg_ok(const asift_pair_cfg &pc)
{
    return pc.kmax >= 0 && pc.kmax <= 7 && pc.ratio_den >= 1 && pc.ratio_num >= 0 && (pc.coarse == 0 || pc.coarse == 1) &&
           (!pc.coarse || (pc.ds >= 0.0 && pc.ds <= 2.0)) &&
           (pc.interp == ASIFT_INTERP_LANCZOS3 || pc.interp == ASIFT_INTERP_NEAREST);
}

static bool pipeline_layout(const asift_ctx *ctx, const PairSpec *ps, int P, const asift_pair_cfg &pc, bool per_view,
                            void *base, Pipeline &L)
{
    const asift_orb_cfg &cfg = ctx->cfg;
    const int N = cfg.n_features;
    L.n_pairs = P;
    L.nv1.assign(P, 0);
    L.nv2.assign(P, 0);
    L.first.assign(2 * P + 1, 0);
    L.views.clear();
    for (int p = 0; p < P; ++p) {
        const int a = pair_views(ps[p], pc, 0, nullptr, 0);
        const int b = pair_views(ps[p], pc, 1, nullptr, 0);
        L.nv1[p] = a;
        L.nv2[p] = b;
        const size_t o = L.views.size();
        L.views.resize(o + a + b);
        pair_views(ps[p], pc, 0, L.views.data() + o, a);
        pair_views(ps[p], pc, 1, L.views.data() + o + a, b);
        L.first[2 * p + 1] = (int)o + a;
        L.first[2 * p + 2] = (int)o + a + b;
    }
    L.nv = (int)L.views.size();
    if (L.nv > 65535 || L.nv < 1) return false;
    // the tables uploaded per call are contiguous: dv, probs, conv, lv, group_first
    Bump b(base);
    L.status = b.take<int32_t>(64);
    const size_t tab0 = (b.off + 255) & ~(size_t)255;
    L.dv = b.take<DevView>(L.nv);
    L.probs = b.take<MatchProblem>(P);
    L.conv = b.take<ImageConv>(2 * P);
    L.grp = b.take<DevRotGroup>(L.nv);
    build_levels(cfg, L.views.data(), L.nv, nullptr, nullptr, nullptr, nullptr, per_view, L.T, ctx->test_cand_cap);
    orb_layout(b, L.T, L.nv, 2 * P, cfg, L.o);
    L.tab_bytes = (size_t)((char *)(L.o.group_first + 2 * P + 1) - (char *)L.dv);
    if (!base) {                              // sizing pass: the same offsets from a null base
        Bump c(nullptr);
        c.take<int32_t>(64);
        c.take<DevView>(L.nv);
        c.take<MatchProblem>(P);
        c.take<ImageConv>(2 * P);
        c.take<DevRotGroup>(L.nv);
        c.take<DevLevel>(std::max<size_t>((size_t)cfg.n_levels * L.nv, 1));
        c.take<int32_t>(2 * P + 1);
        L.tab_bytes = c.off - tab0;
    }
    L.o.status = L.status;
    build_levels(cfg, L.views.data(), L.nv, nullptr, nullptr, L.o.arena_u8, L.o.arena_mask, per_view, L.T,
                 ctx->test_cand_cap);
    L.level0_off.assign(L.nv, 0);
    long long off = 0;
    for (int v = 0; v < L.nv; ++v) {
        L.level0_off[v] = off;
        for (int l = 0; l < cfg.n_levels; ++l)
            off += ((long long)level_size(L.views[v].Wv, l) * level_size(L.views[v].Hv, l) + 15) & ~15LL;
    }
    L.tilt_filters = b.take<float>(std::max<size_t>(tilt_filter_floats(L.views.data(), L.nv), 1));
    L.src.assign(2 * P, nullptr);
    L.max_px = 0;
    for (int p = 0; p < P; ++p) {
        L.src[2 * p] = b.take<float>((size_t)src_pitch_of(ps[p].W1) * ps[p].H1);
        L.src[2 * p + 1] = b.take<float>((size_t)src_pitch_of(ps[p].W2) * ps[p].H2);
        L.max_px = std::max(L.max_px, std::max((long long)ps[p].W1 * ps[p].H1, (long long)ps[p].W2 * ps[p].H2));
    }
    L.view_count = b.take<int32_t>(L.nv);
    L.view_off = b.take<int32_t>(L.nv);
    const size_t cap = (size_t)L.nv * N;
    L.cap_rows = (long long)cap;
    L.n_per_view = N;
    L.kp = b.take<asift_keypoint>(cap);
    L.desc = b.take<uint8_t>(cap * 32);
    L.xdesc = b.take<uint8_t>(tc_expanded_bytes((long long)cap));
    L.match = b.take<asift_match>(cap);
    L.accept = b.take<uint8_t>(cap);
    L.n_acc = b.take<int32_t>(P);
    L.part.assign(P, nullptr);
    L.h_probs.assign(P, MatchProblem{});
    for (int p = 0; p < P; ++p) {
        const int nq = L.nv1[p] * N, nt = L.nv2[p] * N;
        L.part[p] = b.take<unsigned char>(hamming_partial_bytes(nq, nt));
        const size_t q0 = (size_t)L.first[2 * p] * N, t0 = (size_t)L.first[2 * p + 1] * N;
        MatchProblem &M = L.h_probs[p];
        match_problem_init(M, L.desc + q0 * 32, nq, L.o.group_total + 2 * p, L.desc + t0 * 32, nt,
                           L.o.group_total + 2 * p + 1, L.part[p], 0, L.match + q0, L.accept + q0, L.n_acc + p);
        M.kp1 = L.kp + q0;
        M.kp2 = L.kp + t0;
    }
    match_problems_offsets(L.h_probs.data(), P, &L.total_q, &L.total_blk);
    L.block_count = b.take<int32_t>(std::max(L.total_blk, 1));
    L.bytes = b.off + 256;
    return true;
}

// Fills the host tables that depend on the image pointers and the outputs,
// and packs everything that goes to the device into one blob starting at dv.
static void pipeline_tables(Pipeline &L, const asift_pair_desc *pairs, asift_pair_match *const *outs,
                            const int *caps, int32_t *const *d_ns, bool per_view, std::vector<unsigned char> &blob,
                            int seg_w = 0)
{
    const int P = L.n_pairs;
    std::vector<const float *> srcs(L.nv);
    std::vector<int> pitches(L.nv);
    L.h_conv.assign(2 * P, ImageConv{});
    for (int p = 0; p < P; ++p) {
        for (int im = 0; im < 2; ++im) {
            const int g = 2 * p + im;
            for (int v = L.first[g]; v < L.first[g + 1]; ++v) {
                srcs[v] = L.src[g];
                pitches[v] = src_pitch_of(im ? pairs[p].W2 : pairs[p].W1);
            }
            ImageConv &c = L.h_conv[g];
            c.src = im ? pairs[p].d_img2 : pairs[p].d_img1;
            c.dst = L.src[g];
            c.pitch = im ? pairs[p].pitch2 : pairs[p].pitch1;
            c.W = im ? pairs[p].W2 : pairs[p].W1;
            c.H = im ? pairs[p].H2 : pairs[p].H1;
            c.dpitch = src_pitch_of(c.W);
        }
        L.h_probs[p].pairs = outs[p];
        L.h_probs[p].cap = caps[p];
        L.h_probs[p].d_n = d_ns[p];
    }
    build_views(L.views.data(), L.nv, srcs.data(), pitches.data(), L.level0_off.data(), per_view, L.tilt_filters,
                L.h_dv, &L.n_tiles, &L.cw_max, &L.hp_max, &L.max_wv);
    L.seg_w = seg_w > 0 ? seg_w : warp_seg_width_default();
    build_rot_groups(L.views.data(), L.h_dv.data(), L.nv, per_view, L.seg_w, L.h_grp, &L.grp_tiles, &L.hk_max);
    blob.assign(L.tab_bytes, 0);
    char *b0 = (char *)L.dv;
    std::memcpy(blob.data(), L.h_dv.data(), sizeof(DevView) * L.nv);
    std::memcpy(blob.data() + ((char *)L.grp - b0), L.h_grp.data(), sizeof(DevRotGroup) * L.h_grp.size());
    std::memcpy(blob.data() + ((char *)L.o.lv - b0), L.T.lv.data(), sizeof(DevLevel) * L.T.lv.size());
    std::memcpy(blob.data() + ((char *)L.o.group_first - b0), L.first.data(), sizeof(int32_t) * L.first.size());
    std::memcpy(blob.data() + ((char *)L.probs - b0), L.h_probs.data(), sizeof(MatchProblem) * P);
    std::memcpy(blob.data() + ((char *)L.conv - b0), L.h_conv.data(), sizeof(ImageConv) * 2 * P);
}

// The launch sequence (tables already on the device).
static cudaError_t pipeline_run(asift_ctx *ctx, const Pipeline &L, const asift_pair_cfg &pc, bool per_view,
                                const asift_tuning *tune, cudaStream_t s)
{
    const int P = L.n_pairs;
    cudaError_t e = launch_convert_images(L.conv, 2 * P, L.max_px, s);
    prof_mark(ctx, 1, s);
    if (e == cudaSuccess) {
        const bool nearest = pc.interp == ASIFT_INTERP_NEAREST;
        if (!per_view) {
            if (nearest) {
                e = launch_warp_nn(L.dv, L.nv, L.n_tiles, L.cw_max, L.o.arena_u8, L.o.arena_mask, nullptr, s,
                                   tune ? tune->warp_grid : 0);
            } else {
                e = launch_tilt_filter(L.dv, L.nv, L.max_wv, s);
                if (e == cudaSuccess)
                    e = launch_warp(L.grp, (int)L.h_grp.size(), L.dv, L.grp_tiles, L.seg_w, L.hk_max, L.o.arena_u8,
                                    L.o.arena_mask, nullptr, s, tune ? tune->warp_grid : 0);
            }
        } else {
            for (int v = 0; v < L.nv && e == cudaSuccess; ++v) {
                const int tiles = L.h_dv[v].ntx * ((L.views[v].Hv + kWarpTH - 1) / kWarpTH);
                if (nearest) {
                    e = launch_warp_nn(L.dv + v, 1, tiles, L.cw_max, L.o.arena_u8, L.o.arena_mask, nullptr, s);
                    continue;
                }
                e = launch_tilt_filter(L.dv + v, 1, L.views[v].Wv, s);
                const DevRotGroup &g = L.h_grp[v];     // per view: group v is view v alone
                if (e == cudaSuccess)
                    e = launch_warp(L.grp + v, 1, L.dv, g.nseg * g.nbands, L.seg_w, L.hk_max, L.o.arena_u8,
                                    L.o.arena_mask, nullptr, s);
            }
        }
    }
    prof_mark(ctx, 2, s);
    if (e == cudaSuccess)
        e = run_orb(ctx, L.T, L.nv, 2 * P, L.o, per_view, L.kp, L.desc, L.view_count, L.view_off, s, tune);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.n_acc, 0, sizeof(int32_t) * P, s);
    if (e == cudaSuccess) {
        MatchTuning mt{tune ? tune->match_grid : 0, tune ? tune->match_target_items : 0, ctx->test_stall_ns};
        if (resolve_engine(ctx, tune) == ASIFT_MATCH_TENSOR_CORES) {
            if (!tc_match_available()) return cudaErrorNotSupported;
            e = launch_expand(L.desc, L.xdesc, L.o.group_first, L.n_per_view, L.o.group_total, L.cap_rows, 2 * P, s);
            if (e == cudaSuccess)
                e = launch_match_tc(L.desc, L.xdesc, L.cap_rows, L.desc, L.xdesc, L.cap_rows, L.probs, P,
                                    L.h_probs[0], L.total_q, pc.ratio_num, pc.ratio_den, mt, L.status, s);
        } else {
            e = launch_match(L.probs, P, L.h_probs[0], L.total_q, true, pc.ratio_num, pc.ratio_den, mt, s);
        }
    }
    prof_mark(ctx, 7, s);
    if (e == cudaSuccess)
        e = launch_pairs(L.probs, P, L.h_probs[0], L.total_blk, L.block_count, L.o.lv, L.nv, L.status, s);
    prof_mark(ctx, 8, s);
    return e;
}

}  // namespace asift

extern "C" {

static asift_pair_cfg pair_cfg_or_default(const asift_pair_cfg *c)
{
    asift_pair_cfg d{5, 4, 5, 0, 0, ASIFT_INTERP_LANCZOS3, 0.5};
    return c ? *c : d;
}

size_t match_pair_workspace_size(const asift_ctx *ctx, int H1, int W1, int H2, int W2, const asift_pair_cfg *cfg)
{
    if (!ctx || H1 < 1 || W1 < 1 || H2 < 1 || W2 < 1) return 0;
    const asift_pair_cfg pc = pair_cfg_or_default(cfg);
    if (!pair_cfg_ok(pc)) return 0;
    Pipeline L;
    PairSpec ps{H1, W1, H2, W2};
    if (!pipeline_layout(ctx, &ps, 1, pc, pc.per_view != 0, nullptr, L)) return 0;
    return L.bytes;
}

asift_status match_pair(asift_ctx *ctx, const uint8_t *d_img1, int H1, int W1, int pitch1, const uint8_t *d_img2,
                        int H2, int W2, int pitch2, const asift_pair_cfg *cfg, asift_pair_match *d_out, int cap,
                        int32_t *d_n, void *d_workspace, size_t ws_bytes, void *stream)
{
    const asift_pair_cfg pc = pair_cfg_or_default(cfg);
    if (!ctx || !d_img1 || !d_img2 || H1 < 1 || W1 < 1 || H2 < 1 || W2 < 1 || H1 > 16384 || W1 > 16384 ||
        H2 > 16384 || W2 > 16384 || pitch1 < W1 || pitch2 < W2 || !pair_cfg_ok(pc) || cap < 0 ||
        (cap && !d_out) || !d_n || !d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
        return ASIFT_ERR_ARG;
    const bool per_view = pc.per_view != 0;
    const PairKey key{d_img1, d_img2, H1, W1, pitch1, H2, W2, pitch2, pc.kmax, pc.ratio_num, pc.ratio_den,
                      pc.per_view, pc.coarse, pc.interp, pc.ds, d_out, cap, d_n, d_workspace};
    if (!ctx->pair_cache) ctx->pair_cache = new (std::nothrow) PairCache;
    if (!ctx->pair_cache) return ASIFT_ERR_NOMEM;
    PairCache &C = *ctx->pair_cache;
    PairCache::Entry *hit = nullptr;
    for (auto &en : C.e)
        if (en.key == key) hit = &en;
    if (!hit) {
        PairCache::Entry fresh;
        fresh.key = key;
        PairSpec ps{H1, W1, H2, W2};
        if (!pipeline_layout(ctx, &ps, 1, pc, per_view, d_workspace, fresh.L)) return ASIFT_ERR_ARG;
        if (ws_bytes < fresh.L.bytes) return ASIFT_ERR_ARG;
        asift_pair_desc pd{d_img1, H1, W1, pitch1, d_img2, H2, W2, pitch2};
        pipeline_tables(fresh.L, &pd, &d_out, &cap, &d_n, per_view, fresh.blob);
        if (C.e.size() < PairCache::kEntries) {
            C.e.push_back(std::move(fresh));
            hit = &C.e.back();
        } else {
            hit = &C.e[0];
            for (auto &en : C.e)
                if (en.used < hit->used) hit = &en;
            *hit = std::move(fresh);
        }
    }
    hit->used = ++C.clock;
    const Pipeline &L = hit->L;
    if (ws_bytes < L.bytes) return ASIFT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    prof_mark(ctx, 0, s);
    cudaError_t e = upload(ctx, L.dv, hit->blob.data(), hit->blob.size(), s);
    if (e == cudaSuccess) e = pipeline_run(ctx, L, pc, per_view, nullptr, s);
    return cuda_status(e);
}

asift_status match_pair_inspect(const asift_ctx *ctx, int H1, int W1, int H2, int W2, const asift_pair_cfg *cfg,
                                void *d_workspace, asift_keypoint **d_kp1, uint8_t **d_desc1, int32_t **d_n1,
                                asift_keypoint **d_kp2, uint8_t **d_desc2, int32_t **d_n2, asift_match **d_match)
{
    if (!ctx || !d_workspace) return ASIFT_ERR_ARG;
    const asift_pair_cfg pc = pair_cfg_or_default(cfg);
    Pipeline L;
    PairSpec ps{H1, W1, H2, W2};
    if (!pair_cfg_ok(pc) || !pipeline_layout(ctx, &ps, 1, pc, pc.per_view != 0, d_workspace, L)) return ASIFT_ERR_ARG;
    const size_t off2 = (size_t)L.first[1] * ctx->cfg.n_features;
    if (d_kp1) *d_kp1 = L.kp;
    if (d_desc1) *d_desc1 = L.desc;
    if (d_n1) *d_n1 = L.o.group_total;
    if (d_kp2) *d_kp2 = L.kp + off2;
    if (d_desc2) *d_desc2 = L.desc + off2 * 32;
    if (d_n2) *d_n2 = L.o.group_total + 1;
    if (d_match) *d_match = L.match;
    return ASIFT_OK;
}

size_t asift_eval_workspace_size(int cap, int n_hyp)
{
    if (cap < 0 || cap > (1 << 26) || n_hyp < 0 || n_hyp > (1 << 20)) return 0;
    return eval_workspace_bytes(cap, n_hyp);
}

asift_status asift_eval_pairs(asift_ctx *ctx, const asift_pair_match *d_pairs, const int32_t *d_n, int cap,
                              const double *h_H_true, double th_sq, const uint32_t *d_rnd, int n_hyp,
                              double ransac_th_sq, asift_pair_match *d_unique, uint8_t *d_inlier,
                              int32_t *d_hyp_counts, asift_eval_result *d_result, void *d_workspace, size_t ws_bytes,
                              void *stream)
{
    if (!ctx || !d_n || !d_result || !d_workspace || cap < 0 || cap > (1 << 26) || n_hyp < 0 || n_hyp > (1 << 20) ||
        (cap > 0 && (!d_pairs || !d_unique)) || (n_hyp > 0 && !d_rnd) || !(th_sq >= 0.0) ||
        !(ransac_th_sq >= 0.0) || (reinterpret_cast<uintptr_t>(d_workspace) & 255) ||
        ws_bytes < eval_workspace_bytes(cap, n_hyp))
        return ASIFT_ERR_ARG;
    return cuda_status(launch_eval(d_pairs, d_n, cap, h_H_true, th_sq, d_rnd, n_hyp, ransac_th_sq, d_unique, d_inlier,
                                   d_hyp_counts, d_result, d_workspace, static_cast<cudaStream_t>(stream)));
}

size_t asift_sift_match_workspace_size(int nq, int nt)
{
    if (nq < 0 || nt < 0 || nq > (1 << 22) || nt > (1 << 22)) return 0;
    return sift_match_workspace_bytes(nq, nt);
}

asift_status asift_sift_match(asift_ctx *ctx, const float *d_q, int nq, const int32_t *d_nq, const float *d_t, int nt,
                              const int32_t *d_nt, double ratio, const asift_sift_kp *d_kq, const asift_sift_kp *d_kt,
                              asift_l2_match *d_out, asift_pair_match *d_pairs, int cap, int32_t *d_n_pairs,
                              void *d_workspace, size_t ws_bytes, void *stream)
{
    if (!ctx || nq < 0 || nt < 0 || nq > (1 << 22) || nt > (1 << 22) || (nq && (!d_q || !d_out)) || (nt && !d_t) ||
        !(ratio > 0.0 && ratio <= 1.0) || cap < 0 || (d_n_pairs && d_kq && d_kt && cap > 0 && !d_pairs) ||
        !d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255) ||
        (reinterpret_cast<uintptr_t>(d_q) & 15) || (reinterpret_cast<uintptr_t>(d_t) & 15) ||
        ws_bytes < sift_match_workspace_bytes(nq, nt))
        return ASIFT_ERR_ARG;
    return cuda_status(launch_sift_match(d_q, nq, d_nq, d_t, nt, d_nt, ratio, d_kq, d_kt, d_out, d_pairs, cap,
                                         d_n_pairs, d_workspace, static_cast<cudaStream_t>(stream)));
}

size_t asift_sift_workspace_size(int H, int W, int max_kp)
{
    if (H < 16 || W < 16 || H > 16384 || W > 16384 || max_kp < 1 || max_kp > (1 << 20)) return 0;
    return sift_workspace_bytes(W, H, max_kp);
}

asift_status asift_sift(asift_ctx *ctx, const uint8_t *d_img, int H, int W, int pitch, int max_kp, asift_sift_kp *d_kp,
                        float *d_desc, int32_t *d_n, void *d_workspace, size_t ws_bytes, void *stream)
{
    if (!ctx || !d_img || !d_kp || !d_desc || !d_n || !d_workspace || H < 16 || W < 16 || H > 16384 || W > 16384 ||
        pitch < W || max_kp < 1 || max_kp > (1 << 20) || (reinterpret_cast<uintptr_t>(d_workspace) & 255) ||
        ws_bytes < sift_workspace_bytes(W, H, max_kp))
        return ASIFT_ERR_ARG;
    return cuda_status(launch_sift(d_img, W, H, pitch, max_kp, d_kp, d_desc, d_n, d_workspace,
                                   static_cast<cudaStream_t>(stream)));
}

size_t asift_scale_coefficient_workspace_size(int cap)
{
    if (cap < 0 || cap > (1 << 26)) return 0;
    return scale_coeff_workspace_bytes(cap);
}

asift_status asift_scale_coefficient(asift_ctx *ctx, const asift_pair_match *d_pairs, const int32_t *d_n, int cap,
                                     double *d_f, void *d_workspace, size_t ws_bytes, void *stream)
{
    if (!ctx || !d_n || !d_f || !d_workspace || cap < 0 || cap > (1 << 26) || (cap > 0 && !d_pairs) ||
        (reinterpret_cast<uintptr_t>(d_workspace) & 255) || ws_bytes < scale_coeff_workspace_bytes(cap))
        return ASIFT_ERR_ARG;
    return cuda_status(launch_scale_coeff(d_pairs, d_n, cap, d_f, d_workspace, static_cast<cudaStream_t>(stream)));
}

asift_status match_pair_view_counts(asift_ctx *ctx, int H1, int W1, int H2, int W2, const asift_pair_cfg *cfg,
                                    void *d_workspace, int32_t *d_counts, int n_counts, int32_t *d_best, void *stream)
{
    if (!ctx || !d_workspace || !d_counts || n_counts < 1) return ASIFT_ERR_ARG;
    const asift_pair_cfg pc = pair_cfg_or_default(cfg);
    if (!pair_cfg_ok(pc) || pc.per_view) return ASIFT_ERR_ARG;
    Pipeline L;
    PairSpec ps{H1, W1, H2, W2};
    if (!pipeline_layout(ctx, &ps, 1, pc, false, d_workspace, L)) return ASIFT_ERR_ARG;
    const int nv1 = L.nv1[0];
    if (n_counts < nv1 || nv1 > view_count_max_views()) return ASIFT_ERR_ARG;
    return cuda_status(launch_view_counts(L.kp, L.accept, L.o.group_total, L.first[1] * ctx->cfg.n_features,
                                          L.first[0], nv1, d_counts, d_best, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"

// ---------------------------------------------------------------- batched plan
static bool tuning_ok(const asift_tuning &t)
{
    return t.warp_grid >= 0 && t.pyramid_grid >= 0 && t.detect_grid >= 0 && t.match_grid >= 0 &&
           t.match_target_items >= 0 && t.match_engine >= ASIFT_MATCH_AUTO && t.match_engine <= ASIFT_MATCH_TENSOR_CORES &&
           (t.warp_seg == 0 || (t.warp_seg >= 64 && t.warp_seg <= 1024));
}

struct asift_plan {
    asift_ctx *ctx = nullptr;
    asift_pair_cfg pc{};
    asift_tuning tune{};
    std::vector<asift_pair_desc> pairs;
    asift::Pipeline L;
    void *ws = nullptr;
    std::vector<asift_pair_match *> outs;
    std::vector<int> caps;
    int32_t *d_ns = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
};

static void plan_free(asift_plan *p)
{
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto *o : p->outs)
        if (o) cudaFree(o);
    if (p->d_ns) cudaFree(p->d_ns);
    if (p->ws) cudaFree(p->ws);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

// The view simulation's rotation groups for the plan's warp_seg (rebuilt and
// uploaded when it changed).
static cudaError_t plan_regroup(asift_plan *p)
{
    asift::Pipeline &L = p->L;
    const int seg = p->tune.warp_seg > 0 ? p->tune.warp_seg : asift::warp_seg_width_default();
    if (seg == L.seg_w) return cudaSuccess;
    std::vector<DevRotGroup> g;
    int tiles = 0, hk = 3;
    asift::build_rot_groups(L.views.data(), L.h_dv.data(), L.nv, false, seg, g, &tiles, &hk);
    if (!asift::warp_seg_width_ok(seg, hk)) return cudaErrorInvalidValue;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess) e = cudaMemcpy(L.grp, g.data(), sizeof(DevRotGroup) * g.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    L.h_grp.swap(g);
    L.grp_tiles = tiles;
    L.hk_max = hk;
    L.seg_w = seg;
    return cudaSuccess;
}

// Captures the launch sequence of the plan in a CUDA graph on its stream.
static cudaError_t plan_capture(asift_plan *p)
{
    cudaError_t r0 = plan_regroup(p);
    if (r0 != cudaSuccess) return r0;
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    if (!p->use_graph) return cudaSuccess;
    const bool prof = p->ctx->prof;
    p->ctx->prof = false;                    // no stage events inside the graph
    cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t r = asift::pipeline_run(p->ctx, p->L, p->pc, false, &p->tune, p->stream);
        cudaError_t c = cudaStreamEndCapture(p->stream, &p->graph);
        e = (r != cudaSuccess) ? r : c;
    }
    p->ctx->prof = prof;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    return e;
}

static cudaError_t plan_launch(asift_plan *p, cudaStream_t s)
{
    if (p->use_graph && p->exec) return cudaGraphLaunch(p->exec, s);
    return asift::pipeline_run(p->ctx, p->L, p->pc, false, &p->tune, s);
}

extern "C" {

asift_status asift_plan_create(asift_ctx *ctx, const asift_pair_desc *h_pairs, int n_pairs,
                               const asift_pair_cfg *cfg, const asift_tuning *tuning, int use_graph,
                               asift_plan **out)
{
    if (!ctx || !h_pairs || n_pairs < 1 || n_pairs > asift::match_max_problems() || !out) return ASIFT_ERR_ARG;
    *out = nullptr;
    const asift_pair_cfg pc = pair_cfg_or_default(cfg);
    if (!pair_cfg_ok(pc) || pc.per_view) return ASIFT_ERR_ARG;
    if (tuning && !tuning_ok(*tuning)) return ASIFT_ERR_ARG;
    std::vector<asift::PairSpec> ps(n_pairs);
    for (int i = 0; i < n_pairs; ++i) {
        const asift_pair_desc &d = h_pairs[i];
        if (!d.d_img1 || !d.d_img2 || d.H1 < 1 || d.W1 < 1 || d.H2 < 1 || d.W2 < 1 || d.H1 > 16384 || d.W1 > 16384 ||
            d.H2 > 16384 || d.W2 > 16384 || d.pitch1 < d.W1 || d.pitch2 < d.W2)
            return ASIFT_ERR_ARG;
        ps[i] = asift::PairSpec{d.H1, d.W1, d.H2, d.W2};
    }
    asift_plan *p = new (std::nothrow) asift_plan;
    if (!p) return ASIFT_ERR_NOMEM;
    p->ctx = ctx;
    p->pc = pc;
    if (tuning) p->tune = *tuning;
    p->use_graph = use_graph != 0;
    p->pairs.assign(h_pairs, h_pairs + n_pairs);
    if (!asift::pipeline_layout(ctx, ps.data(), n_pairs, pc, false, nullptr, p->L)) {
        plan_free(p);
        return ASIFT_ERR_ARG;
    }
    const size_t bytes = p->L.bytes;
    if (cudaMalloc(&p->ws, bytes) != cudaSuccess) { plan_free(p); return ASIFT_ERR_NOMEM; }
    if (cudaMemset(p->ws, 0, 256) != cudaSuccess) { plan_free(p); return ASIFT_ERR_CUDA; }
    p->L = asift::Pipeline{};
    asift::pipeline_layout(ctx, ps.data(), n_pairs, pc, false, p->ws, p->L);
    p->outs.assign(n_pairs, nullptr);
    p->caps.assign(n_pairs, 0);
    if (cudaMalloc(&p->d_ns, sizeof(int32_t) * n_pairs) != cudaSuccess) { plan_free(p); return ASIFT_ERR_NOMEM; }
    std::vector<int32_t *> ns(n_pairs);
    for (int i = 0; i < n_pairs; ++i) {
        p->caps[i] = std::max(1, p->L.nv1[i] * ctx->cfg.n_features);
        if (cudaMalloc(&p->outs[i], sizeof(asift_pair_match) * p->caps[i]) != cudaSuccess) {
            plan_free(p);
            return ASIFT_ERR_NOMEM;
        }
        ns[i] = p->d_ns + i;
    }
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
        plan_free(p);
        return ASIFT_ERR_CUDA;
    }
    std::vector<unsigned char> blob;
    asift::pipeline_tables(p->L, p->pairs.data(), p->outs.data(), p->caps.data(), ns.data(), false, blob,
                           p->tune.warp_seg);
    if (!asift::warp_seg_width_ok(p->L.seg_w, p->L.hk_max)) {
        plan_free(p);
        return ASIFT_ERR_ARG;
    }
    cudaError_t e = cudaMemcpyAsync(p->L.dv, blob.data(), blob.size(), cudaMemcpyHostToDevice, p->stream);
    // one plain run validates the sequence and sets the kernels' attributes before capture
    if (e == cudaSuccess) e = asift::pipeline_run(ctx, p->L, pc, false, &p->tune, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess) e = plan_capture(p);
    if (e != cudaSuccess) {
        plan_free(p);
        return ASIFT_ERR_CUDA;
    }
    *out = p;
    return ASIFT_OK;
}

asift_status asift_plan_run(asift_plan *plan, void *stream)
{
    if (!plan) return ASIFT_ERR_ARG;
    return cuda_status(plan_launch(plan, static_cast<cudaStream_t>(stream)));
}

asift_status asift_plan_pairs(const asift_plan *plan, int i, asift_pair_match **d_pairs, int *cap, int32_t **d_n)
{
    if (!plan || i < 0 || i >= (int)plan->outs.size()) return ASIFT_ERR_ARG;
    if (d_pairs) *d_pairs = plan->outs[i];
    if (cap) *cap = plan->caps[i];
    if (d_n) *d_n = plan->d_ns + i;
    return ASIFT_OK;
}

asift_status asift_plan_view_counts(const asift_plan *plan, int i, int32_t *d_counts, int n_counts, int32_t *d_best,
                                    void *stream)
{
    if (!plan || i < 0 || i >= (int)plan->outs.size() || !d_counts) return ASIFT_ERR_ARG;
    const asift::Pipeline &L = plan->L;
    const int nv1 = L.nv1[i];
    if (n_counts < nv1 || nv1 > view_count_max_views()) return ASIFT_ERR_ARG;
    const size_t q0 = (size_t)L.first[2 * i] * plan->ctx->cfg.n_features;
    return cuda_status(launch_view_counts(L.kp + q0, L.accept + q0, L.o.group_total + 2 * i,
                                          nv1 * plan->ctx->cfg.n_features, L.first[2 * i], nv1, d_counts, d_best,
                                          static_cast<cudaStream_t>(stream)));
}

size_t asift_plan_eval_workspace_size(const asift_plan *plan, int n_hyp)
{
    if (!plan || n_hyp < 0 || n_hyp > (1 << 20)) return 0;
    return eval_batch_workspace_bytes(plan->caps.data(), (int)plan->caps.size(), n_hyp);
}

asift_status asift_plan_eval(asift_plan *plan, const double *h_H_true, double th_sq, const uint32_t *d_rnd, int n_hyp,
                             double ransac_th_sq, void *d_workspace, size_t ws_bytes, void *stream)
{
    if (!plan || !d_workspace || n_hyp < 0 || n_hyp > (1 << 20) || (n_hyp > 0 && !d_rnd) || !(th_sq >= 0.0) ||
        !(ransac_th_sq >= 0.0) || (reinterpret_cast<uintptr_t>(d_workspace) & 255) ||
        ws_bytes < eval_batch_workspace_bytes(plan->caps.data(), (int)plan->caps.size(), n_hyp))
        return ASIFT_ERR_ARG;
    return cuda_status(launch_eval_batch(plan->outs.data(), plan->d_ns, plan->caps.data(), (int)plan->caps.size(),
                                         h_H_true, th_sq, d_rnd, n_hyp, ransac_th_sq, d_workspace,
                                         static_cast<cudaStream_t>(stream)));
}

asift_status asift_plan_eval_outputs(const asift_plan *plan, void *d_workspace, int n_hyp, int i,
                                     asift_pair_match **d_unique, uint8_t **d_inlier, int32_t **d_hyp_counts,
                                     asift_eval_result **d_result)
{
    if (!plan || !d_workspace || i < 0 || i >= (int)plan->caps.size() || n_hyp < 0 || n_hyp > (1 << 20))
        return ASIFT_ERR_ARG;
    eval_batch_outputs(d_workspace, plan->caps.data(), (int)plan->caps.size(), n_hyp, i, d_unique, d_inlier,
                       d_hyp_counts, d_result);
    return ASIFT_OK;
}

asift_status asift_plan_workspace(const asift_plan *plan, void **d_workspace, int32_t **d_pool_counts)
{
    if (!plan) return ASIFT_ERR_ARG;
    if (d_workspace) *d_workspace = plan->ws;
    if (d_pool_counts) *d_pool_counts = plan->L.o.group_total;
    return ASIFT_OK;
}

asift_status asift_plan_set_tuning(asift_plan *plan, const asift_tuning *tuning)
{
    if (!plan || !tuning) return ASIFT_ERR_ARG;
    if (!tuning_ok(*tuning)) return ASIFT_ERR_ARG;
    const asift_tuning old = plan->tune;
    plan->tune = *tuning;
    if (cudaStreamSynchronize(plan->stream) != cudaSuccess) return ASIFT_ERR_CUDA;
    const cudaError_t e = plan_capture(plan);
    if (e == cudaErrorInvalidValue) {           // a tile shape the views do not fit
        plan->tune = old;
        plan_capture(plan);
        return ASIFT_ERR_ARG;
    }
    return cuda_status(e);
}

asift_status asift_plan_get_tuning(const asift_plan *plan, asift_tuning *out)
{
    if (!plan || !out) return ASIFT_ERR_ARG;
    *out = plan->tune;
    return ASIFT_OK;
}

// Milliseconds per replay of the plan's current sequence.
static cudaError_t plan_time(asift_plan *p, int reps, float *ms)
{
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) { cudaEventDestroy(a); return e; }
    e = plan_launch(p, p->stream);                 // warm
    if (e == cudaSuccess) e = cudaEventRecord(a, p->stream);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = plan_launch(p, p->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b, p->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (e == cudaSuccess) *ms /= std::max(1, reps);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

asift_status asift_plan_autotune(asift_plan *plan, int reps, asift_tuning *out)
{
    if (!plan || reps < 1) return ASIFT_ERR_ARG;
    const int sms = asift::device_sm_count();
    // coordinate descent over one knob at a time, the others at their best
    struct Knob {
        int32_t *field;
        std::vector<int> cands;
    };
    asift_tuning &t = plan->tune;
    std::vector<Knob> knobs = {
        {&t.warp_seg, {0, 384, 512, 768}},     // the view simulation's tile shape (0 = 576)
        {&t.warp_grid, {0, 3 * sms, 4 * sms}},
        {&t.pyramid_grid, {0, 4 * sms, 8 * sms}},
        {&t.detect_grid, {0, 8 * sms, 16 * sms}},
    };
    if (tc_match_available()) knobs.push_back({&t.match_engine, {ASIFT_MATCH_TENSOR_CORES, ASIFT_MATCH_CUDA_CORES}});
    cudaError_t e = cudaSuccess;
    auto tune_knob = [&](const Knob &k) {
        int best = *k.field;
        float best_ms = 1e30f;
        for (int c : k.cands) {
            *k.field = c;
            e = plan_capture(plan);
            if (e == cudaErrorInvalidValue) {      // a tile shape these views do not fit: skipped
                cudaGetLastError();
                e = cudaSuccess;
                continue;
            }
            float ms = 0.f;
            if (e == cudaSuccess) e = plan_time(plan, reps, &ms);
            if (e != cudaSuccess) break;
            if (ms < best_ms) { best_ms = ms; best = c; }
        }
        *k.field = best;
    };
    for (const Knob &k : knobs) {
        tune_knob(k);
        if (e != cudaSuccess) break;
    }
    // the matcher's launch shape, for the engine chosen above
    std::vector<Knob> mk;
    if (resolve_engine(plan->ctx, &t) == ASIFT_MATCH_TENSOR_CORES) {
        t.match_grid = 0;                                   // one CTA per SM
        mk.push_back({&t.match_target_items, {0, 4 * sms, 8 * sms, 24 * sms}});   // 0: 12 x SMs
    } else {
        mk.push_back({&t.match_grid, {7 * sms, 4 * sms}});
        mk.push_back({&t.match_target_items, {0, 4 * 7 * sms, 7 * sms}});
    }
    for (const Knob &k : mk) {
        if (e != cudaSuccess) break;
        tune_knob(k);
    }
    if (e == cudaSuccess) e = plan_capture(plan);
    if (out) *out = plan->tune;
    return cuda_status(e);
}

void asift_plan_destroy(asift_plan *plan) { plan_free(plan); }

}  // extern "C"

// ---------------------------------------------------------------- differentiable warp
extern "C" {

asift_status asift_warp_shape_for(int H, int W, double t0, double phi0, double t_max, asift_warp_shape *out)
{
    if (H < 1 || W < 1 || H > 16384 || W > 16384 || !(t0 >= 1.0 && t0 < 11.4) || !(t_max >= t0 && t_max < 11.4) ||
        !out || !(phi0 == phi0))
        return ASIFT_ERR_ARG;
    asift_view_desc v;
    make_view_desc(H, W, t0, phi0, -1, -1, 1.0, &v);
    out->Wr = v.Wr;
    out->Hr = v.Hr;
    out->Wv = v.Wv;
    out->Hv = v.Hv;
    out->K = (int32_t)std::ceil(4.0 * (t_max > 1.0 ? 0.8 * std::sqrt(t_max * t_max - 1.0) : 0.0));
    out->pad = 0;
    if (out->K >= ASIFT_MAX_GAUSS) return ASIFT_ERR_ARG;
    return ASIFT_OK;
}

size_t asift_warp_workspace_size(int n)
{
    Bump b(nullptr);
    b.take<int32_t>(64);
    b.take<DiffView>(std::max(n, 1));
    b.take<DiffPrep>(std::max(n, 1));
    return b.off + 256;
}

static asift_status warp_call(bool backward, asift_ctx *ctx, const float *d_u, int H, int W, int n,
                              const double *d_params, const asift_warp_shape *h_shapes, double t_max,
                              float *d_v, const float *d_vbar, const int64_t *h_voff, float *d_ubar, double *d_pbar,
                              void *d_ws, size_t ws_bytes, void *stream)
{
    if (!ctx || !d_u || H < 1 || W < 1 || n < 1 || !d_params || !h_shapes || !h_voff || !d_ws ||
        !(t_max >= 1.0 && t_max < 11.4) || (!backward && !d_v) || (backward && (!d_vbar || !d_pbar)))
        return ASIFT_ERR_ARG;
    if (ws_bytes < asift_warp_workspace_size(n)) return ASIFT_ERR_ARG;
    Bump b(d_ws);
    int32_t *status = b.take<int32_t>(64);
    DiffView *tab = b.take<DiffView>(n);
    DiffPrep *prep = b.take<DiffPrep>(n);
    std::vector<DiffView> h(n);
    int tiles = 0, cw_max = 1, bw_max = 1;
    for (int i = 0; i < n; ++i) {
        const asift_warp_shape &S = h_shapes[i];
        if (S.Wr < 1 || S.Hr < 1 || S.Wv < 1 || S.Hv < 1 || S.K < 0 || S.K >= ASIFT_MAX_GAUSS || h_voff[i] < 0)
            return ASIFT_ERR_ARG;
        DiffView &d = h[i];
        d = DiffView{};
        d.u = d_u + (size_t)i * H * W;
        d.ubar = (backward && d_ubar) ? d_ubar + (size_t)i * H * W : nullptr;
        d.vbar = backward ? d_vbar + h_voff[i] : nullptr;
        d.out = backward ? nullptr : d_v + h_voff[i];
        d.param = d_params + 4 * (size_t)i;
        d.pbar = backward ? d_pbar + 4 * (size_t)i : nullptr;
        d.W = W;
        d.H = H;
        d.Wr = S.Wr;
        d.Hr = S.Hr;
        d.Wv = S.Wv;
        d.Hv = S.Hv;
        d.K = S.K;
        d.tile_start = tiles;
        d.tw = dwarp_tile_width(backward);
        tiles += dwarp_tiles(S.Wv, S.Hv, d.tw, &d.ntx);
        int cw, bw;
        dwarp_strip_widths(d.tw, t_max, S.K, &cw, &bw);
        cw_max = std::max(cw_max, cw);
        bw_max = std::max(bw_max, bw);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = upload(ctx, tab, h.data(), sizeof(DiffView) * n, s);
    if (e == cudaSuccess && backward && d_ubar) e = cudaMemsetAsync(d_ubar, 0, sizeof(float) * (size_t)n * H * W, s);
    if (e == cudaSuccess && backward) e = cudaMemsetAsync(d_pbar, 0, sizeof(double) * 4 * (size_t)n, s);
    if (e == cudaSuccess) e = launch_dwarp(backward, tab, prep, n, tiles, cw_max, bw_max, status, s);
    return cuda_status(e);
}

asift_status asift_warp_fwd(asift_ctx *ctx, const float *d_u, int H, int W, int n, const double *d_params,
                            const asift_warp_shape *h_shapes, double t_max, float *d_v, const int64_t *h_voff,
                            void *d_workspace, size_t ws_bytes, void *stream)
{
    return warp_call(false, ctx, d_u, H, W, n, d_params, h_shapes, t_max, d_v, nullptr, h_voff, nullptr, nullptr,
                     d_workspace, ws_bytes, stream);
}

asift_status asift_warp_bwd(asift_ctx *ctx, const float *d_u, int H, int W, int n, const double *d_params,
                            const asift_warp_shape *h_shapes, double t_max, const float *d_vbar, const int64_t *h_voff,
                            float *d_ubar, double *d_pbar, void *d_workspace, size_t ws_bytes, void *stream)
{
    return warp_call(true, ctx, d_u, H, W, n, d_params, h_shapes, t_max, nullptr, d_vbar, h_voff, d_ubar, d_pbar,
                     d_workspace, ws_bytes, stream);
}

asift_status asift_warp_loss(asift_ctx *ctx, int n, const asift_warp_shape *h_shapes, const int64_t *h_voff,
                             const float *d_v, const float *d_target, double *d_loss, float *d_vbar, void *d_workspace,
                             size_t ws_bytes, void *stream)
{
    if (!ctx || n < 1 || !h_shapes || !h_voff || !d_v || !d_target || !d_loss || !d_workspace ||
        ws_bytes < asift_warp_workspace_size(n))
        return ASIFT_ERR_ARG;
    Bump b(d_workspace);
    b.take<int32_t>(64);
    WarpSeg *tab = reinterpret_cast<WarpSeg *>(b.take<DiffView>(n));   // the view table's room holds the segments
    std::vector<WarpSeg> h(n);
    long long mx = 0;
    for (int i = 0; i < n; ++i) {
        if (h_shapes[i].Wv < 1 || h_shapes[i].Hv < 1 || h_voff[i] < 0) return ASIFT_ERR_ARG;
        h[i].off = h_voff[i];
        h[i].count = (long long)h_shapes[i].Wv * h_shapes[i].Hv;
        mx = std::max(mx, h[i].count);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = upload(ctx, tab, h.data(), sizeof(WarpSeg) * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_loss, 0, sizeof(double) * n, s);
    if (e == cudaSuccess) e = launch_warp_loss(tab, n, mx, d_v, d_target, d_loss, d_vbar, s);
    return cuda_status(e);
}

asift_status asift_warp_adam(asift_ctx *ctx, int n, double *d_params, const double *d_grad, double *d_m, double *d_v,
                             int step, const double *h_lr, double decay, double t_lo, double t_hi, void *stream)
{
    if (!ctx || n < 1 || !d_params || !d_grad || !d_m || !d_v || step < 0 || !h_lr || !(decay > 0.0) ||
        !(t_lo >= 1.0 && t_lo <= t_hi && t_hi < 11.4))
        return ASIFT_ERR_ARG;
    AdamArgs a{};
    for (int k = 0; k < 4; ++k) a.lr[k] = h_lr[k];
    a.scale = std::pow(decay, (double)step);
    a.c1 = 1.0 - std::pow(0.9, (double)step + 1);
    a.c2 = 1.0 - std::pow(0.999, (double)step + 1);
    a.t_lo = t_lo;
    a.t_hi = t_hi;
    return cuda_status(launch_warp_adam(n, d_params, d_grad, d_m, d_v, a, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
