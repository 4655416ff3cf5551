// sift.cu -- SIFT (Lowe 2004) for the precise stage (Sec. III-C: SIFT on the
// Lanczos reproduction of the best view against the target) on sm_103a, fp32.
//
//   1. base_kernel: the 8-bit image / 255 doubled by centre-aligned bilinear
//      interpolation;
//   2. blur_h_kernel / blur_v_kernel: separable Gaussian (taps from the host,
//      radius floor(4 sigma + 1/2), edge pixels replicated) for the initial
//      blur to sigma0 = 1.6 and the S + 2 incremental blurs of each octave;
//      half_kernel starts an octave from image S of the previous one;
//      dog_kernel takes the differences;
//   3. extrema_kernel: one thread per pixel of DoG layers 1..S: the contrast
//      prefilter, the strict 26-neighbour test, the quadratic refinement (at
//      most 5 moves), the contrast and edge tests; survivors are appended;
//   4. orient_kernel: one thread per candidate: the 36-bin gradient histogram,
//      smoothing, peaks within 80% of the highest, parabolic refinement;
//      keypoints are appended (one per peak);
//   5. sift_desc_kernel: one CTA per keypoint: the 4 x 4 x 8 histogram of
//      the rotated window in shared memory (trilinear spreading), normalised,
//      clamped at 0.2, renormalised.
// The keypoint order is that of the appends; callers sort by response.  The
// descriptor sums are shared-memory float atomics: their last bits depend on
// the order of the adds.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace asift {

constexpr int kSiftS = 3;
constexpr int kSiftLayers = kSiftS + 3;
constexpr int kSiftMaxOct = 12;
constexpr int kSiftMaxTaps = 64;
constexpr float kSiftSigma0 = 1.6f;
constexpr float kSiftContrast = 0.04f;
constexpr float kSiftEdgeR = 10.f;
constexpr int kSiftBorder = 5;
constexpr int kSiftOriBins = 36;
constexpr int kSiftDescThreads = 128;

struct SiftTaps {
    int r;
    float g[kSiftMaxTaps];
};

struct SiftPyr {
    int n_oct;
    int W[kSiftMaxOct], H[kSiftMaxOct];
    float *G[kSiftMaxOct][kSiftLayers];
    float *D[kSiftMaxOct][kSiftLayers - 1];
};

struct SiftCand {
    float xo, yo, s, contrast;
    int o, k;
};

__global__ void base_kernel(const uint8_t *__restrict__ img, int pitch, int W, int H, float *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    const int W2 = 2 * W, H2 = 2 * H;
    if (x >= W2 || y >= H2) return;
    const float sx = (x + 0.5f) * 0.5f - 0.5f, sy = (y + 0.5f) * 0.5f - 0.5f;
    const int x0 = (int)floorf(sx), y0 = (int)floorf(sy);
    const float fx = sx - x0, fy = sy - y0;
    const int xa = clampi(x0, 0, W - 1), xb = clampi(x0 + 1, 0, W - 1);
    const int ya = clampi(y0, 0, H - 1), yb = clampi(y0 + 1, 0, H - 1);
    const float k = 1.0f / 255.0f;
    const float a = img[(size_t)ya * pitch + xa] * k, b = img[(size_t)ya * pitch + xb] * k;
    const float c = img[(size_t)yb * pitch + xa] * k, d = img[(size_t)yb * pitch + xb] * k;
    const float top = (1.f - fx) * a + fx * b, bot = (1.f - fx) * c + fx * d;
    out[(size_t)y * W2 + x] = (1.f - fy) * top + fy * bot;
}

__global__ void blur_h_kernel(const float *__restrict__ src, int W, int H, const SiftTaps T, float *__restrict__ dst)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const float *row = src + (size_t)y * W;
    float acc = 0.f;
    for (int k = -T.r; k <= T.r; ++k) acc = fmaf(T.g[k + T.r], row[clampi(x + k, 0, W - 1)], acc);
    dst[(size_t)y * W + x] = acc;
}

__global__ void blur_v_kernel(const float *__restrict__ src, int W, int H, const SiftTaps T, float *__restrict__ dst)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    float acc = 0.f;
    for (int k = -T.r; k <= T.r; ++k) acc = fmaf(T.g[k + T.r], src[(size_t)clampi(y + k, 0, H - 1) * W + x], acc);
    dst[(size_t)y * W + x] = acc;
}

__global__ void half_kernel(const float *__restrict__ src, int Ws, float *__restrict__ dst, int W, int H)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    dst[(size_t)y * W + x] = src[(size_t)(2 * y) * Ws + 2 * x];
}

__global__ void dog_kernel(const float *__restrict__ a, const float *__restrict__ b, float *__restrict__ d, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = b[i] - a[i];
}

__device__ __forceinline__ float pat(const float *p, int W, int x, int y) { return p[(size_t)y * W + x]; }

// 3x3 solve by Gaussian elimination with partial pivoting; false if singular.
__device__ bool solve3f(float A[3][3], float b[3], float x[3])
{
    for (int c = 0; c < 3; ++c) {
        int p = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabsf(A[r][c]) > fabsf(A[p][c])) p = r;
        if (!(fabsf(A[p][c]) > 1e-30f)) return false;
        if (p != c) {
            for (int k = 0; k < 3; ++k) {
                const float t = A[c][k];
                A[c][k] = A[p][k];
                A[p][k] = t;
            }
            const float t = b[c];
            b[c] = b[p];
            b[p] = t;
        }
        for (int r = c + 1; r < 3; ++r) {
            const float f = A[r][c] / A[c][c];
            for (int k = c; k < 3; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        float s = b[r];
        for (int k = r + 1; k < 3; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return true;
}

// grid (x, y, layer 1..S) of one octave
__global__ void extrema_kernel(const SiftPyr P, int o, SiftCand *__restrict__ cand, int cap, int *__restrict__ n_cand)
{
    const int W = P.W[o], H = P.H[o];
    int x = blockIdx.x * blockDim.x + threadIdx.x + kSiftBorder, y = blockIdx.y * blockDim.y + threadIdx.y + kSiftBorder;
    int k = blockIdx.z + 1;
    if (x >= W - kSiftBorder || y >= H - kSiftBorder) return;
    const float v0 = pat(P.D[o][k], W, x, y);
    if (!(fabsf(v0) > 0.5f * kSiftContrast / kSiftS)) return;
    bool is_max = true, is_min = true;
    for (int dk = -1; dk <= 1; ++dk)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dk && !dy && !dx) continue;
                const float w = pat(P.D[o][k + dk], W, x + dx, y + dy);
                if (!(v0 > w)) is_max = false;
                if (!(v0 < w)) is_min = false;
            }
    if (!is_max && !is_min) return;
    float off[3], g[3], dxx = 0.f, dyy = 0.f, dxy = 0.f, contrast = 0.f;
    bool ok = false;
    for (int it = 0; it < 5; ++it) {
        const float *c = P.D[o][k], *pr = P.D[o][k - 1], *nx = P.D[o][k + 1];
        const float v = pat(c, W, x, y);
        g[0] = (pat(c, W, x + 1, y) - pat(c, W, x - 1, y)) * 0.5f;
        g[1] = (pat(c, W, x, y + 1) - pat(c, W, x, y - 1)) * 0.5f;
        g[2] = (pat(nx, W, x, y) - pat(pr, W, x, y)) * 0.5f;
        dxx = pat(c, W, x + 1, y) + pat(c, W, x - 1, y) - 2.f * v;
        dyy = pat(c, W, x, y + 1) + pat(c, W, x, y - 1) - 2.f * v;
        const float dss = pat(nx, W, x, y) + pat(pr, W, x, y) - 2.f * v;
        dxy = (pat(c, W, x + 1, y + 1) - pat(c, W, x - 1, y + 1) - pat(c, W, x + 1, y - 1) + pat(c, W, x - 1, y - 1)) *
              0.25f;
        const float dxs = (pat(nx, W, x + 1, y) - pat(nx, W, x - 1, y) - pat(pr, W, x + 1, y) + pat(pr, W, x - 1, y)) *
                          0.25f;
        const float dys = (pat(nx, W, x, y + 1) - pat(nx, W, x, y - 1) - pat(pr, W, x, y + 1) + pat(pr, W, x, y - 1)) *
                          0.25f;
        float A[3][3] = {{dxx, dxy, dxs}, {dxy, dyy, dys}, {dxs, dys, dss}};
        float b[3] = {-g[0], -g[1], -g[2]};
        if (!solve3f(A, b, off)) return;
        if (fabsf(off[0]) < 0.5f && fabsf(off[1]) < 0.5f && fabsf(off[2]) < 0.5f) {
            contrast = v + 0.5f * (g[0] * off[0] + g[1] * off[1] + g[2] * off[2]);
            ok = true;
            break;
        }
        if (fabsf(off[0]) > 1e6f || fabsf(off[1]) > 1e6f || fabsf(off[2]) > 1e6f) return;
        x += __float2int_rn(off[0]);
        y += __float2int_rn(off[1]);
        k += __float2int_rn(off[2]);
        if (k < 1 || k > kSiftS || x < kSiftBorder || x >= W - kSiftBorder || y < kSiftBorder || y >= H - kSiftBorder)
            return;
    }
    if (!ok || fabsf(contrast) < kSiftContrast / kSiftS) return;
    const float tr = dxx + dyy, det = dxx * dyy - dxy * dxy;
    if (det <= 0.f || tr * tr * kSiftEdgeR >= (kSiftEdgeR + 1.f) * (kSiftEdgeR + 1.f) * det) return;
    const int slot = atomicAdd(n_cand, 1);
    if (slot >= cap) return;
    SiftCand cd;
    cd.xo = x + off[0];
    cd.yo = y + off[1];
    cd.s = kSiftSigma0 * exp2f((k + off[2]) / kSiftS);
    cd.contrast = contrast;
    cd.o = o;
    cd.k = k;
    cand[slot] = cd;
}

__device__ __forceinline__ void gradf(const float *G, int W, int x, int y, float *gx, float *gy)
{
    *gx = pat(G, W, x + 1, y) - pat(G, W, x - 1, y);
    *gy = pat(G, W, x, y + 1) - pat(G, W, x, y - 1);
}

__global__ void orient_kernel(const SiftPyr P, const SiftCand *__restrict__ cand, const int *__restrict__ n_cand,
                              int cap_cand, asift_sift_kp *__restrict__ kps, int cap, int *__restrict__ n_kp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(*n_cand, cap_cand)) return;
    const SiftCand c = cand[i];
    const int W = P.W[c.o], H = P.H[c.o];
    const float *G = P.G[c.o][c.k];
    float h[kSiftOriBins], hs[kSiftOriBins];
    for (int b = 0; b < kSiftOriBins; ++b) h[b] = 0.f;
    const float sig = 1.5f * c.s;
    const int rad = __float2int_rn(3.0f * sig);
    const int cx = __float2int_rn(c.xo), cy = __float2int_rn(c.yo);
    for (int dy = -rad; dy <= rad; ++dy)
        for (int dx = -rad; dx <= rad; ++dx) {
            const int x = cx + dx, y = cy + dy;
            if (x <= 0 || x >= W - 1 || y <= 0 || y >= H - 1) continue;
            float gx, gy;
            gradf(G, W, x, y, &gx, &gy);
            float a = atan2f(gy, gx) * (180.0f / 3.14159265358979f);
            if (a < 0.f) a += 360.f;
            const float w = __expf(-(float)(dx * dx + dy * dy) / (2.f * sig * sig));
            int b = __float2int_rn(a * kSiftOriBins / 360.f);
            b = ((b % kSiftOriBins) + kSiftOriBins) % kSiftOriBins;
            h[b] += w * sqrtf(gx * gx + gy * gy);
        }
    float mx = 0.f;
    for (int b = 0; b < kSiftOriBins; ++b) {
        const int m1 = (b + kSiftOriBins - 1) % kSiftOriBins, m2 = (b + kSiftOriBins - 2) % kSiftOriBins;
        const int p1 = (b + 1) % kSiftOriBins, p2 = (b + 2) % kSiftOriBins;
        hs[b] = (h[m2] + h[p2]) * (1.f / 16.f) + (h[m1] + h[p1]) * (4.f / 16.f) + h[b] * (6.f / 16.f);
        mx = fmaxf(mx, hs[b]);
    }
    const float scale = ldexpf(1.f, c.o);
    for (int b = 0; b < kSiftOriBins; ++b) {
        const float l = hs[(b + kSiftOriBins - 1) % kSiftOriBins], r = hs[(b + 1) % kSiftOriBins];
        if (!(hs[b] > l && hs[b] > r && hs[b] >= 0.8f * mx && mx > 0.f)) continue;
        const float bb = b + 0.5f * (l - r) / (l - 2.f * hs[b] + r);
        float a = fmodf(bb * 360.f / kSiftOriBins + 360.f, 360.f);
        const int slot = atomicAdd(n_kp, 1);
        if (slot >= cap) continue;
        asift_sift_kp k;
        k.x = (c.xo * scale + 0.5f) * 0.5f - 0.5f;
        k.y = (c.yo * scale + 0.5f) * 0.5f - 0.5f;
        k.sigma = c.s * scale * 0.5f;
        k.angle = a;
        k.response = fabsf(c.contrast);
        k.octave = c.o;
        k.layer = c.k;
        k.xo = c.xo;
        k.yo = c.yo;
        k.so = c.s;
        kps[slot] = k;
    }
}

// one CTA per keypoint
__global__ void __launch_bounds__(kSiftDescThreads)
sift_desc_kernel(const SiftPyr P, const asift_sift_kp *__restrict__ kps, const int *__restrict__ n_kp, int cap,
                 float *__restrict__ desc)
{
    constexpr int D = 4, N = 8;
    __shared__ float hist[(D + 2) * (D + 2) * (N + 2)];
    __shared__ float red[kSiftDescThreads];
    const int i = blockIdx.x;
    if (i >= min(*n_kp, cap)) return;
    const asift_sift_kp kp = kps[i];
    for (int t = threadIdx.x; t < (D + 2) * (D + 2) * (N + 2); t += blockDim.x) hist[t] = 0.f;
    __syncthreads();
    const int W = P.W[kp.octave], H = P.H[kp.octave];
    const float *G = P.G[kp.octave][kp.layer];
    const float t = kp.angle * (3.14159265358979f / 180.f);
    float st, ct;
    sincosf(t, &st, &ct);
    const float hw = 3.0f * kp.so;
    const int rad = __float2int_rn(hw * 1.41421356f * (D + 1) * 0.5f);
    const int cx = __float2int_rn(kp.xo), cy = __float2int_rn(kp.yo);
    const float wsig = 0.5f * D;
    const int side = 2 * rad + 1;
    for (int s = threadIdx.x; s < side * side; s += blockDim.x) {
        const int dy = s / side - rad, dx = s % side - rad;
        const float c_rot = (dx * ct + dy * st) / hw, r_rot = (-dx * st + dy * ct) / hw;
        const float rbin = r_rot + D / 2.f - 0.5f, cbin = c_rot + D / 2.f - 0.5f;
        if (!(rbin > -1.f && rbin < D && cbin > -1.f && cbin < D)) continue;
        const int x = cx + dx, y = cy + dy;
        if (x <= 0 || x >= W - 1 || y <= 0 || y >= H - 1) continue;
        float gx, gy;
        gradf(G, W, x, y, &gx, &gy);
        float a = atan2f(gy, gx) - t;
        while (a < 0.f) a += 6.28318530717959f;
        while (a >= 6.28318530717959f) a -= 6.28318530717959f;
        const float obin = a * N / 6.28318530717959f;
        const float mag = sqrtf(gx * gx + gy * gy) * __expf(-(c_rot * c_rot + r_rot * r_rot) / (2.f * wsig * wsig));
        const int r0 = (int)floorf(rbin), c0 = (int)floorf(cbin), o0 = min((int)floorf(obin), N - 1);
        const float fr = rbin - r0, fc = cbin - c0, fo = obin - o0;
        for (int ir = 0; ir <= 1; ++ir)
            for (int ic = 0; ic <= 1; ++ic)
                for (int io = 0; io <= 1; ++io) {
                    const float w = (ir ? fr : 1.f - fr) * (ic ? fc : 1.f - fc) * (io ? fo : 1.f - fo);
                    const int rr = r0 + ir + 1, cc = c0 + ic + 1, oo = (o0 + io) % N;
                    atomicAdd(&hist[(rr * (D + 2) + cc) * (N + 2) + oo], w * mag);
                }
    }
    __syncthreads();
    // 128 threads, one bin each
    const int b = threadIdx.x;
    const int r = b / (D * N), c = (b / N) % D, ob = b % N;
    float v = hist[((r + 1) * (D + 2) + (c + 1)) * (N + 2) + ob];
    red[b] = v * v;
    __syncthreads();
    for (int w = kSiftDescThreads / 2; w > 0; w >>= 1) {
        if (b < w) red[b] += red[b + w];
        __syncthreads();
    }
    const float nrm = sqrtf(red[0]);
    __syncthreads();
    v = nrm > 0.f ? fminf(v / nrm, 0.2f) : 0.f;
    red[b] = v * v;
    __syncthreads();
    for (int w = kSiftDescThreads / 2; w > 0; w >>= 1) {
        if (b < w) red[b] += red[b + w];
        __syncthreads();
    }
    const float n2 = sqrtf(red[0]);
    desc[(size_t)i * 128 + b] = n2 > 0.f ? v / n2 : 0.f;
}

// ---------------------------------------------------------------- host side
static SiftTaps gauss_taps_host(double sigma)
{
    SiftTaps T{};
    T.r = std::min((int)(4.0 * sigma + 0.5), (kSiftMaxTaps - 1) / 2);
    double g[kSiftMaxTaps], sum = 0.0;
    for (int k = -T.r; k <= T.r; ++k) {
        g[k + T.r] = std::exp(-(double)(k * k) / (2.0 * sigma * sigma));
        sum += g[k + T.r];
    }
    for (int k = 0; k <= 2 * T.r; ++k) T.g[k] = (float)(g[k] / sum);
    return T;
}

static int sift_octaves(int W, int H)
{
    const int mn = std::min(2 * W, 2 * H);
    return std::max(1, std::min(kSiftMaxOct, (int)std::floor(std::log2((double)mn)) - 3));
}

static size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// Workspace: the tmp image, every octave's Gaussians and DoGs, candidates, counters.
static size_t sift_layout(int W, int H, int max_kp, char *base, SiftPyr *P, float **tmp, SiftCand **cand,
                          int *cap_cand, int **counters)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    const int n_oct = sift_octaves(W, H);
    if (P) P->n_oct = n_oct;
    int w = 2 * W, h = 2 * H;
    float *t = reinterpret_cast<float *>(take(sizeof(float) * (size_t)w * h));
    if (tmp) *tmp = t;
    for (int o = 0; o < n_oct; ++o) {
        if (o > 0) {
            w /= 2;
            h /= 2;
        }
        if (P) {
            P->W[o] = w;
            P->H[o] = h;
        }
        for (int k = 0; k < kSiftLayers; ++k) {
            float *g = reinterpret_cast<float *>(take(sizeof(float) * (size_t)w * h));
            if (P) P->G[o][k] = g;
        }
        for (int k = 0; k < kSiftLayers - 1; ++k) {
            float *d = reinterpret_cast<float *>(take(sizeof(float) * (size_t)w * h));
            if (P) P->D[o][k] = d;
        }
    }
    // candidates: far more than images give (a fraction of the doubled image's
    // pixels), and at least max_kp
    const int cc = std::max(max_kp, (int)std::min<long long>((long long)W * H / 2 + 1024, 1LL << 24));
    SiftCand *c = reinterpret_cast<SiftCand *>(take(sizeof(SiftCand) * (size_t)cc));
    if (cand) *cand = c;
    if (cap_cand) *cap_cand = cc;
    int *cnt = reinterpret_cast<int *>(take(sizeof(int) * 4));
    if (counters) *counters = cnt;
    return off;
}

size_t sift_workspace_bytes(int W, int H, int max_kp)
{
    return sift_layout(W, H, max_kp, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

cudaError_t launch_sift(const uint8_t *d_img, int W, int H, int pitch, int max_kp, asift_sift_kp *d_kp, float *d_desc,
                        int32_t *d_n, void *d_ws, cudaStream_t s)
{
    SiftPyr P{};
    float *tmp;
    SiftCand *cand;
    int cap_cand, *cnt;
    sift_layout(W, H, max_kp, static_cast<char *>(d_ws), &P, &tmp, &cand, &cap_cand, &cnt);
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * 4, s);
    if (e != cudaSuccess) return e;
    const dim3 blk(32, 8);
    auto grid2 = [&](int w, int h) { return dim3((w + 31) / 32, (h + 7) / 8); };
    int launches = 0;
    // base and its blur to sigma0 from an assumed 2 x 0.5
    base_kernel<<<grid2(2 * W, 2 * H), blk, 0, s>>>(d_img, pitch, W, H, tmp);
    const double s_in = 1.0;
    const SiftTaps T0 = gauss_taps_host(std::sqrt(std::max(1.6 * 1.6 - s_in * s_in, 0.01)));
    blur_h_kernel<<<grid2(P.W[0], P.H[0]), blk, 0, s>>>(tmp, P.W[0], P.H[0], T0, P.G[0][1]);
    blur_v_kernel<<<grid2(P.W[0], P.H[0]), blk, 0, s>>>(P.G[0][1], P.W[0], P.H[0], T0, P.G[0][0]);
    launches += 3;
    for (int o = 0; o < P.n_oct; ++o) {
        const int w = P.W[o], h = P.H[o];
        if (o > 0) {
            half_kernel<<<grid2(w, h), blk, 0, s>>>(P.G[o - 1][kSiftS], P.W[o - 1], P.G[o][0], w, h);
            ++launches;
        }
        for (int k = 1; k < kSiftLayers; ++k) {
            const double sp = 1.6 * std::pow(2.0, (double)(k - 1) / kSiftS), st = 1.6 * std::pow(2.0, (double)k / kSiftS);
            const SiftTaps T = gauss_taps_host(std::sqrt(st * st - sp * sp));
            blur_h_kernel<<<grid2(w, h), blk, 0, s>>>(P.G[o][k - 1], w, h, T, tmp);
            blur_v_kernel<<<grid2(w, h), blk, 0, s>>>(tmp, w, h, T, P.G[o][k]);
            launches += 2;
        }
        for (int k = 0; k < kSiftLayers - 1; ++k) {
            const int n = w * h;
            dog_kernel<<<(n + 255) / 256, 256, 0, s>>>(P.G[o][k], P.G[o][k + 1], P.D[o][k], n);
            ++launches;
        }
    }
    for (int o = 0; o < P.n_oct; ++o) {
        const int iw = P.W[o] - 2 * kSiftBorder, ih = P.H[o] - 2 * kSiftBorder;
        if (iw <= 0 || ih <= 0) continue;
        extrema_kernel<<<dim3((iw + 31) / 32, (ih + 7) / 8, kSiftS), blk, 0, s>>>(P, o, cand, cap_cand, cnt);
        ++launches;
    }
    orient_kernel<<<(cap_cand + 127) / 128, 128, 0, s>>>(P, cand, cnt, cap_cand, d_kp, max_kp, cnt + 1);
    sift_desc_kernel<<<std::max(1, max_kp), kSiftDescThreads, 0, s>>>(P, d_kp, cnt + 1, max_kp, d_desc);
    launches += 2;
    note_launch(launches);
    e = cudaMemcpyAsync(d_n, cnt + 1, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace asift
