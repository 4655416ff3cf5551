/*
 * sift_oracle.c -- plain, slow CPU oracle of SIFT (Lowe, "Distinctive image
 * features from scale-invariant keypoints", IJCV 2004), the detector and
 * descriptor of the precise stage of arXiv 2503.03479 (Sec. III-C: SIFT on
 * the Lanczos reproduction of the best view against the target).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it shares no code, header or table with the CUDA path.
 *
 * fp64 throughout, single-threaded, scalar.  The steps follow Lowe's paper in
 * its order (the paper under study names SIFT without details):
 *   1. scale space: the image (grey levels / 255) doubled by centre-aligned
 *      bilinear interpolation, blurred to sigma0 = 1.6 from an assumed 2 x 0.5;
 *      S = 3 intervals per octave, S + 3 Gaussian images per octave, each
 *      octave starting from image S of the previous one subsampled by 2;
 *      difference-of-Gaussian images;
 *   2. extrema of the DoG over their 26 neighbours in layers 1..S, 5 px from
 *      the border, |D| > 0.5 * 0.04 / S;
 *   3. refinement by the 3-D quadratic fit (at most 5 moves), rejection of
 *      low contrast (|D(x^)| < 0.04 / S) and of edges (tr^2 / det >= 11^2 / 10);
 *   4. orientations: a 36-bin histogram of gradient directions (Gaussian
 *      window 1.5 sigma, radius 3 x 1.5 sigma), smoothed, every peak within
 *      80% of the highest, refined by a parabola;
 *   5. descriptor: 4 x 4 x 8 histograms over a window rotated to the
 *      orientation (bin width 3 sigma, Gaussian weight of half the window,
 *      trilinear spreading), unit-normalised, clamped at 0.2, renormalised;
 *   6. brute-force L2 matching with the ratio test (in fp64, and with its
 *      decisions taken in fp32 in a fixed order, as the GPU takes them).
 * Angles are those of the image gradient (gx, gy) with x to the right and y
 * down: atan2(gy, gx) in degrees, in [0, 360).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SIFT_S 3
#define SIFT_SIGMA0 1.6
#define SIFT_INIT_BLUR 0.5
#define SIFT_CONTRAST 0.04
#define SIFT_EDGE_R 10.0
#define SIFT_BORDER 5
#define SIFT_MAX_INTERP 5
#define SIFT_ORI_BINS 36
#define SIFT_ORI_SIG 1.5
#define SIFT_ORI_RADIUS 3.0
#define SIFT_ORI_PEAK 0.8
#define SIFT_D 4
#define SIFT_N 8
#define SIFT_HIST_SCL 3.0
#define SIFT_MAG_THR 0.2
#define SIFT_MAX_OCT 12

typedef struct {
    double x, y;        /* original image coordinates                        */
    double sigma;       /* scale in original image pixels                    */
    double angle;       /* degrees, [0, 360)                                 */
    double response;    /* |D| at the refined extremum                       */
    int32_t octave, layer;
} oracle_sift_kp;

typedef struct {
    int W, H;
    double *p;
} simg;

static simg simg_new(int W, int H)
{
    simg a = {W, H, (double *)calloc((size_t)W * H, sizeof(double))};
    return a;
}

static inline int clampi_s(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static inline double px_at(const simg *a, int x, int y) { return a->p[(size_t)y * a->W + x]; }

/* Separable Gaussian blur with taps exp(-k^2 / 2 sigma^2), k = -r..r,
 * r = (int)(4 sigma + 0.5), normalised to sum 1; borders replicate the edge
 * pixel.  dst may not alias src. */
void oracle_gauss_blur(const double *src, int W, int H, double sigma, double *dst)
{
    const int r = (int)(4.0 * sigma + 0.5);
    double *g = (double *)malloc(sizeof(double) * (2 * r + 1));
    double sum = 0.0;
    for (int k = -r; k <= r; ++k) {
        g[k + r] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        sum += g[k + r];
    }
    for (int k = 0; k <= 2 * r; ++k) g[k] /= sum;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)W * H);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int k = -r; k <= r; ++k) acc += g[k + r] * src[(size_t)y * W + clampi_s(x + k, 0, W - 1)];
            tmp[(size_t)y * W + x] = acc;
        }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int k = -r; k <= r; ++k) acc += g[k + r] * tmp[(size_t)clampi_s(y + k, 0, H - 1) * W + x];
            dst[(size_t)y * W + x] = acc;
        }
    free(tmp);
    free(g);
}

/* Twice the size, centre-aligned bilinear: output pixel i samples the input
 * at (i + 1/2) / 2 - 1/2, edge taps clamped. */
static simg upsample2(const simg *a)
{
    simg b = simg_new(2 * a->W, 2 * a->H);
    for (int y = 0; y < b.H; ++y) {
        const double sy = (y + 0.5) / 2.0 - 0.5;
        const int y0 = (int)floor(sy);
        const double fy = sy - y0;
        for (int x = 0; x < b.W; ++x) {
            const double sx = (x + 0.5) / 2.0 - 0.5;
            const int x0 = (int)floor(sx);
            const double fx = sx - x0;
            const int xa = clampi_s(x0, 0, a->W - 1), xb = clampi_s(x0 + 1, 0, a->W - 1);
            const int ya = clampi_s(y0, 0, a->H - 1), yb = clampi_s(y0 + 1, 0, a->H - 1);
            const double top = (1.0 - fx) * px_at(a, xa, ya) + fx * px_at(a, xb, ya);
            const double bot = (1.0 - fx) * px_at(a, xa, yb) + fx * px_at(a, xb, yb);
            b.p[(size_t)y * b.W + x] = (1.0 - fy) * top + fy * bot;
        }
    }
    return b;
}

/* Every second pixel: output (i, j) = input (2i, 2j). */
static simg downsample2(const simg *a)
{
    simg b = simg_new(a->W / 2, a->H / 2);
    for (int y = 0; y < b.H; ++y)
        for (int x = 0; x < b.W; ++x) b.p[(size_t)y * b.W + x] = px_at(a, 2 * x, 2 * y);
    return b;
}

typedef struct {
    int n_oct;
    simg G[SIFT_MAX_OCT][SIFT_S + 3];
    simg D[SIFT_MAX_OCT][SIFT_S + 2];
} pyramid;

static void build_pyramid(const uint8_t *img, int W, int H, pyramid *P)
{
    simg in = simg_new(W, H);
    for (size_t i = 0; i < (size_t)W * H; ++i) in.p[i] = img[i] / 255.0;
    simg up = upsample2(&in);
    free(in.p);
    const double s_in = 2.0 * SIFT_INIT_BLUR;
    const double s_diff = sqrt(fmax(SIFT_SIGMA0 * SIFT_SIGMA0 - s_in * s_in, 0.01));
    simg base = simg_new(up.W, up.H);
    oracle_gauss_blur(up.p, up.W, up.H, s_diff, base.p);
    free(up.p);
    const int mn = up.W < up.H ? up.W : up.H;
    int n_oct = (int)floor(log2((double)mn)) - 3;
    if (n_oct < 1) n_oct = 1;
    if (n_oct > SIFT_MAX_OCT) n_oct = SIFT_MAX_OCT;
    P->n_oct = n_oct;
    for (int o = 0; o < n_oct; ++o) {
        P->G[o][0] = o == 0 ? base : downsample2(&P->G[o - 1][SIFT_S]);
        for (int k = 1; k < SIFT_S + 3; ++k) {
            const double sp = SIFT_SIGMA0 * pow(2.0, (double)(k - 1) / SIFT_S);
            const double st = SIFT_SIGMA0 * pow(2.0, (double)k / SIFT_S);
            const simg *prev = &P->G[o][k - 1];
            P->G[o][k] = simg_new(prev->W, prev->H);
            oracle_gauss_blur(prev->p, prev->W, prev->H, sqrt(st * st - sp * sp), P->G[o][k].p);
        }
        for (int k = 0; k < SIFT_S + 2; ++k) {
            const simg *a = &P->G[o][k], *b = &P->G[o][k + 1];
            P->D[o][k] = simg_new(a->W, a->H);
            for (size_t i = 0; i < (size_t)a->W * a->H; ++i) P->D[o][k].p[i] = b->p[i] - a->p[i];
        }
    }
}

static void free_pyramid(pyramid *P)
{
    for (int o = 0; o < P->n_oct; ++o) {
        for (int k = 0; k < SIFT_S + 3; ++k) free(P->G[o][k].p);
        for (int k = 0; k < SIFT_S + 2; ++k) free(P->D[o][k].p);
    }
}

static int is_extremum(const pyramid *P, int o, int k, int x, int y)
{
    const double v = px_at(&P->D[o][k], x, y);
    int is_max = 1, is_min = 1;
    for (int dk = -1; dk <= 1; ++dk)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dk && !dy && !dx) continue;
                const double w = px_at(&P->D[o][k + dk], x + dx, y + dy);
                if (!(v > w)) is_max = 0;
                if (!(v < w)) is_min = 0;
            }
    return is_max || is_min;
}

/* Solves the 3x3 system A x = b by Gaussian elimination with partial
 * pivoting; 0 if singular. */
static int solve3(double A[3][3], double b[3], double x[3])
{
    for (int c = 0; c < 3; ++c) {
        int p = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        if (fabs(A[p][c]) < 1e-300) return 0;
        if (p != c) {
            for (int k = 0; k < 3; ++k) {
                const double t = A[c][k];
                A[c][k] = A[p][k];
                A[p][k] = t;
            }
            const double t = b[c];
            b[c] = b[p];
            b[p] = t;
        }
        for (int r = c + 1; r < 3; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 3; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < 3; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return 1;
}

/* Step 3: refinement, contrast and edge tests.  On success fills the
 * octave-relative position (xo, yo), layer and layer offset and |D^|. */
/* Margin bookkeeping for the parity tests (does not change any decision):
 * *half receives the smallest distance of an offset component, at any
 * iteration, to the half-integer where its decision (stay, or move by
 * lround) would change; *why the failed test (1 not converged or left the
 * octave, 2 contrast, 3 edge). */
static int refine_ex(const pyramid *P, int o, int *pk, int *px, int *py, double off[3], double *contrast,
                     double *dxx_, double *dyy_, double *dxy_, double *half, int *why);

static int refine(const pyramid *P, int o, int *pk, int *px, int *py, double off[3], double *contrast, double *dxx_,
                  double *dyy_, double *dxy_)
{
    double half;
    int why;
    return refine_ex(P, o, pk, px, py, off, contrast, dxx_, dyy_, dxy_, &half, &why);
}

static double half_dist(double v)
{
    const double a = fabs(v);
    return fabs(a - (floor(a) + 0.5));
}

static int refine_ex(const pyramid *P, int o, int *pk, int *px, int *py, double off[3], double *contrast,
                     double *dxx_, double *dyy_, double *dxy_, double *half, int *why)
{
    int k = *pk, x = *px, y = *py;
    double g[3], Hm[3][3];
    int ok = 0;
    *half = INFINITY;
    *why = 1;
    for (int it = 0; it < SIFT_MAX_INTERP; ++it) {
        const simg *c = &P->D[o][k], *pr = &P->D[o][k - 1], *nx = &P->D[o][k + 1];
        const double v = px_at(c, x, y);
        g[0] = (px_at(c, x + 1, y) - px_at(c, x - 1, y)) * 0.5;
        g[1] = (px_at(c, x, y + 1) - px_at(c, x, y - 1)) * 0.5;
        g[2] = (px_at(nx, x, y) - px_at(pr, x, y)) * 0.5;
        const double dxx = px_at(c, x + 1, y) + px_at(c, x - 1, y) - 2.0 * v;
        const double dyy = px_at(c, x, y + 1) + px_at(c, x, y - 1) - 2.0 * v;
        const double dss = px_at(nx, x, y) + px_at(pr, x, y) - 2.0 * v;
        const double dxy = (px_at(c, x + 1, y + 1) - px_at(c, x - 1, y + 1) - px_at(c, x + 1, y - 1) +
                            px_at(c, x - 1, y - 1)) * 0.25;
        const double dxs = (px_at(nx, x + 1, y) - px_at(nx, x - 1, y) - px_at(pr, x + 1, y) + px_at(pr, x - 1, y)) *
                           0.25;
        const double dys = (px_at(nx, x, y + 1) - px_at(nx, x, y - 1) - px_at(pr, x, y + 1) + px_at(pr, x, y - 1)) *
                           0.25;
        Hm[0][0] = dxx; Hm[0][1] = dxy; Hm[0][2] = dxs;
        Hm[1][0] = dxy; Hm[1][1] = dyy; Hm[1][2] = dys;
        Hm[2][0] = dxs; Hm[2][1] = dys; Hm[2][2] = dss;
        double A[3][3], b[3] = {-g[0], -g[1], -g[2]};
        memcpy(A, Hm, sizeof(A));
        if (!solve3(A, b, off)) return 0;
        for (int q = 0; q < 3; ++q) *half = fmin(*half, half_dist(off[q]));
        if (fabs(off[0]) < 0.5 && fabs(off[1]) < 0.5 && fabs(off[2]) < 0.5) {
            *contrast = v + 0.5 * (g[0] * off[0] + g[1] * off[1] + g[2] * off[2]);
            *dxx_ = dxx;
            *dyy_ = dyy;
            *dxy_ = dxy;
            ok = 1;
            break;
        }
        if (fabs(off[0]) > 1e6 || fabs(off[1]) > 1e6 || fabs(off[2]) > 1e6) return 0;
        x += (int)lround(off[0]);
        y += (int)lround(off[1]);
        k += (int)lround(off[2]);
        if (k < 1 || k > SIFT_S || x < SIFT_BORDER || x >= c->W - SIFT_BORDER || y < SIFT_BORDER ||
            y >= c->H - SIFT_BORDER)
            return 0;
    }
    if (!ok) return 0;
    *pk = k;          /* the refined position, also when a test below fails */
    *px = x;
    *py = y;
    *why = 2;
    if (fabs(*contrast) < SIFT_CONTRAST / SIFT_S) return 0;
    *why = 3;
    const double tr = *dxx_ + *dyy_, det = *dxx_ * *dyy_ - *dxy_ * *dxy_;
    if (det <= 0.0 || tr * tr * SIFT_EDGE_R >= (SIFT_EDGE_R + 1.0) * (SIFT_EDGE_R + 1.0) * det) return 0;
    *why = 0;
    return 1;
}

/* Gradient of a Gaussian image at an interior pixel (central differences). */
static inline void grad(const simg *G, int x, int y, double *gx, double *gy)
{
    *gx = px_at(G, x + 1, y) - px_at(G, x - 1, y);
    *gy = px_at(G, x, y + 1) - px_at(G, x, y - 1);
}

/* Step 4: the orientation histogram of a keypoint at octave-relative (xo,
 * yo) with octave-relative scale s on Gaussian image G.  Returns the number
 * of peaks written to ang[] (degrees). */
static int orientations_ex(const simg *G, double xo, double yo, double s, double *ang, double *margin,
                           double *near_ang, int *n_near, double M);

static int orientations(const simg *G, double xo, double yo, double s, double *ang)
{
    double margin;
    int n_near = 0;
    return orientations_ex(G, xo, yo, s, ang, &margin, NULL, &n_near, 0.0);
}

/* As orientations; *margin = the smallest, over the 36 bins, of |min(h - l,
 * h - r, h - 0.8 max)| / max (a bin is a peak iff that minimum is >= 0 with
 * the first two > 0), and the bins rejected by less than M (relative) go to
 * near_ang[] (when not NULL): for the parity tests, no decision changes. */
static int orientations_ex(const simg *G, double xo, double yo, double s, double *ang, double *margin,
                           double *near_ang, int *n_near, double M)
{
    double h[SIFT_ORI_BINS] = {0}, hs[SIFT_ORI_BINS];
    const double sig = SIFT_ORI_SIG * s;
    const int rad = (int)lround(SIFT_ORI_RADIUS * sig);
    const int cx = (int)lround(xo), cy = (int)lround(yo);
    for (int dy = -rad; dy <= rad; ++dy)
        for (int dx = -rad; dx <= rad; ++dx) {
            const int x = cx + dx, y = cy + dy;
            if (x <= 0 || x >= G->W - 1 || y <= 0 || y >= G->H - 1) continue;
            double gx, gy;
            grad(G, x, y, &gx, &gy);
            double a = atan2(gy, gx) * (180.0 / M_PI);
            if (a < 0.0) a += 360.0;
            const double w = exp(-(double)(dx * dx + dy * dy) / (2.0 * sig * sig));
            int b = (int)lround(a * SIFT_ORI_BINS / 360.0);
            b = ((b % SIFT_ORI_BINS) + SIFT_ORI_BINS) % SIFT_ORI_BINS;
            h[b] += w * sqrt(gx * gx + gy * gy);
        }
    for (int i = 0; i < SIFT_ORI_BINS; ++i) {
        const int m1 = (i + SIFT_ORI_BINS - 1) % SIFT_ORI_BINS, m2 = (i + SIFT_ORI_BINS - 2) % SIFT_ORI_BINS;
        const int p1 = (i + 1) % SIFT_ORI_BINS, p2 = (i + 2) % SIFT_ORI_BINS;
        hs[i] = (h[m2] + h[p2]) * (1.0 / 16.0) + (h[m1] + h[p1]) * (4.0 / 16.0) + h[i] * (6.0 / 16.0);
    }
    double mx = 0.0;
    for (int i = 0; i < SIFT_ORI_BINS; ++i) mx = fmax(mx, hs[i]);
    int n = 0;
    *margin = INFINITY;
    for (int i = 0; i < SIFT_ORI_BINS; ++i) {
        const double l = hs[(i + SIFT_ORI_BINS - 1) % SIFT_ORI_BINS], r = hs[(i + 1) % SIFT_ORI_BINS];
        if (mx > 0.0) {
            const double d = fmin(fmin(hs[i] - l, hs[i] - r), hs[i] - SIFT_ORI_PEAK * mx) / mx;
            *margin = fmin(*margin, fabs(d));
            if (near_ang && d < 0.0 && -d <= M) near_ang[(*n_near)++] = i * 360.0 / SIFT_ORI_BINS;
        }
        if (hs[i] > l && hs[i] > r && hs[i] >= SIFT_ORI_PEAK * mx && mx > 0.0) {
            const double b = i + 0.5 * (l - r) / (l - 2.0 * hs[i] + r);
            double a = b * 360.0 / SIFT_ORI_BINS;
            a = fmod(a + 360.0, 360.0);
            ang[n++] = a;
        }
    }
    return n;
}

/* Step 5: the 4 x 4 x 8 descriptor at octave-relative (xo, yo), scale s,
 * orientation ang (degrees).  A sample's offset is rotated by -ang into the
 * descriptor frame, so the orientation maps to the frame's +x axis. */
static void descriptor(const simg *G, double xo, double yo, double s, double ang, float *out)
{
    double hist[(SIFT_D + 2) * (SIFT_D + 2) * (SIFT_N + 2)];
    memset(hist, 0, sizeof(hist));
    const double t = ang * (M_PI / 180.0);
    const double ct = cos(t), st = sin(t);
    const double hw = SIFT_HIST_SCL * s;
    const int rad = (int)lround(hw * sqrt(2.0) * (SIFT_D + 1) * 0.5);
    const int cx = (int)lround(xo), cy = (int)lround(yo);
    const double wsig = 0.5 * SIFT_D;
    for (int dy = -rad; dy <= rad; ++dy)
        for (int dx = -rad; dx <= rad; ++dx) {
            const double c_rot = (dx * ct + dy * st) / hw, r_rot = (-dx * st + dy * ct) / hw;
            const double rbin = r_rot + SIFT_D / 2.0 - 0.5, cbin = c_rot + SIFT_D / 2.0 - 0.5;
            if (!(rbin > -1.0 && rbin < SIFT_D && cbin > -1.0 && cbin < SIFT_D)) continue;
            const int x = cx + dx, y = cy + dy;
            if (x <= 0 || x >= G->W - 1 || y <= 0 || y >= G->H - 1) continue;
            double gx, gy;
            grad(G, x, y, &gx, &gy);
            double a = atan2(gy, gx) - t;
            while (a < 0.0) a += 2.0 * M_PI;
            while (a >= 2.0 * M_PI) a -= 2.0 * M_PI;
            const double obin = a * SIFT_N / (2.0 * M_PI);
            const double mag = sqrt(gx * gx + gy * gy) * exp(-(c_rot * c_rot + r_rot * r_rot) / (2.0 * wsig * wsig));
            const int r0 = (int)floor(rbin), c0 = (int)floor(cbin), o0 = (int)floor(obin);
            const double fr = rbin - r0, fc = cbin - c0, fo = obin - o0;
            for (int ir = 0; ir <= 1; ++ir)
                for (int ic = 0; ic <= 1; ++ic)
                    for (int io = 0; io <= 1; ++io) {
                        const double w = (ir ? fr : 1.0 - fr) * (ic ? fc : 1.0 - fc) * (io ? fo : 1.0 - fo);
                        const int rr = r0 + ir + 1, cc = c0 + ic + 1, oo = (o0 + io) % SIFT_N;
                        hist[((size_t)rr * (SIFT_D + 2) + cc) * (SIFT_N + 2) + oo] += w * mag;
                    }
        }
    double v[SIFT_D * SIFT_D * SIFT_N];
    double nrm = 0.0;
    for (int r = 0; r < SIFT_D; ++r)
        for (int c = 0; c < SIFT_D; ++c)
            for (int o = 0; o < SIFT_N; ++o) {
                const double e = hist[((size_t)(r + 1) * (SIFT_D + 2) + (c + 1)) * (SIFT_N + 2) + o];
                v[(r * SIFT_D + c) * SIFT_N + o] = e;
                nrm += e * e;
            }
    nrm = sqrt(nrm);
    double n2 = 0.0;
    for (int i = 0; i < SIFT_D * SIFT_D * SIFT_N; ++i) {
        v[i] = nrm > 0.0 ? fmin(v[i] / nrm, SIFT_MAG_THR) : 0.0;
        n2 += v[i] * v[i];
    }
    n2 = sqrt(n2);
    for (int i = 0; i < SIFT_D * SIFT_D * SIFT_N; ++i) out[i] = (float)(n2 > 0.0 ? v[i] / n2 : 0.0);
}

static int kp_cmp(const void *pa, const void *pb)
{
    const oracle_sift_kp *a = (const oracle_sift_kp *)pa, *b = (const oracle_sift_kp *)pb;
    if (a->response != b->response) return a->response > b->response ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    return a->angle < b->angle ? -1 : (a->angle > b->angle);
}

typedef struct {
    oracle_sift_kp kp;
    double xo, yo, s;
    int o, k;
    double margin;      /* smallest relative decision margin (parity tests) */
} kp_full;

static int kpf_cmp(const void *pa, const void *pb) { return kp_cmp(&((const kp_full *)pa)->kp, &((const kp_full *)pb)->kp); }

/* SIFT keypoints and descriptors of an 8-bit image (pitch W).  The
 * strongest max_kp keypoints (|D| descending, then y, x, angle) are written
 * to kps[] and desc[] (128 floats each); returns their number. */
int oracle_sift_ex(const uint8_t *img, int W, int H, int max_kp, oracle_sift_kp *kps, float *desc, double *margin,
                   double *miss, int max_miss, int *n_miss, double M);

int oracle_sift(const uint8_t *img, int W, int H, int max_kp, oracle_sift_kp *kps, float *desc)
{
    return oracle_sift_ex(img, W, H, max_kp, kps, desc, NULL, NULL, 0, NULL, 0.0);
}

/* A near miss, in original image coordinates: (x, y, sigma, angle or -1). */
static void add_miss(double *miss, int max_miss, int *n_miss, int o, double xo, double yo, double s, double ang)
{
    if (!miss || !n_miss || *n_miss >= max_miss) return;
    const double scale = ldexp(1.0, o);
    double *m = miss + 4 * (size_t)(*n_miss)++;
    m[0] = (xo * scale + 0.5) / 2.0 - 0.5;
    m[1] = (yo * scale + 0.5) / 2.0 - 0.5;
    m[2] = s * scale / 2.0;
    m[3] = ang;
}

/* oracle_sift with, for the parity tests (no decision changes): margin[i],
 * the smallest relative margin by which keypoint i passed each of its tests
 * (the pre-threshold, the 26 extremum comparisons, the refinement's rounding
 * decisions, contrast, edge ratio and its orientation bins), and miss[] (4
 * doubles each: x, y, sigma, angle or -1), the candidates rejected by one of
 * those tests by no more than M relative (a near threshold, a near extremum,
 * an offset near a half-integer, a near peak bin). */
int oracle_sift_ex(const uint8_t *img, int W, int H, int max_kp, oracle_sift_kp *kps, float *desc, double *margin,
                   double *miss, int max_miss, int *n_miss, double M)
{
    if (n_miss) *n_miss = 0;
    pyramid *P = (pyramid *)calloc(1, sizeof(pyramid));
    build_pyramid(img, W, H, P);
    int cap = 1024, n = 0;
    kp_full *all = (kp_full *)malloc(sizeof(kp_full) * cap);
    const double pre = 0.5 * SIFT_CONTRAST / SIFT_S;
    for (int o = 0; o < P->n_oct; ++o)
        for (int k = 1; k <= SIFT_S; ++k) {
            const simg *Dk = &P->D[o][k];
            for (int y = SIFT_BORDER; y < Dk->H - SIFT_BORDER; ++y)
                for (int x = SIFT_BORDER; x < Dk->W - SIFT_BORDER; ++x) {
                    const double v = px_at(Dk, x, y);
                    const double s0 = SIFT_SIGMA0 * pow(2.0, (double)k / SIFT_S);
                    if (!(fabs(v) > pre)) {
                        if (fabs(v) > pre * (1.0 - M)) add_miss(miss, max_miss, n_miss, o, x, y, s0, -1.0);
                        continue;
                    }
                    double ext = INFINITY;      /* extremum margin: the closest neighbour, relative to |v| */
                    if (margin || miss) {
                        double hi = -INFINITY, lo = INFINITY;
                        for (int dk = -1; dk <= 1; ++dk)
                            for (int dy = -1; dy <= 1; ++dy)
                                for (int dx = -1; dx <= 1; ++dx) {
                                    if (!dk && !dy && !dx) continue;
                                    const double w = px_at(&P->D[o][k + dk], x + dx, y + dy);
                                    hi = fmax(hi, w);
                                    lo = fmin(lo, w);
                                }
                        ext = fmin(fabs(v - hi), fabs(v - lo)) / fabs(v);
                    }
                    if (!is_extremum(P, o, k, x, y)) {
                        if (ext <= M) add_miss(miss, max_miss, n_miss, o, x, y, s0, -1.0);
                        continue;
                    }
                    int kk = k, xx = x, yy = y;
                    double off[3], contrast, dxx, dyy, dxy, half;
                    int why;
                    const int ok = refine_ex(P, o, &kk, &xx, &yy, off, &contrast, &dxx, &dyy, &dxy, &half, &why);
                    double con_m = INFINITY, edge_m = INFINITY;
                    if (why == 0 || why == 2 || why == 3) {
                        con_m = fabs(fabs(contrast) - SIFT_CONTRAST / SIFT_S) / (SIFT_CONTRAST / SIFT_S);
                        const double tr = dxx + dyy, det = dxx * dyy - dxy * dxy;
                        const double lim = (SIFT_EDGE_R + 1.0) * (SIFT_EDGE_R + 1.0) * det;
                        edge_m = det > 0.0 ? fabs(lim - tr * tr * SIFT_EDGE_R) / lim : 0.0;
                    }
                    if (!ok) {
                        const double m = why == 1 ? half : (why == 2 ? con_m : edge_m);
                        if (m <= M) {
                            const double sk = SIFT_SIGMA0 * pow(2.0, (double)kk / SIFT_S);
                            add_miss(miss, max_miss, n_miss, o, xx, yy, sk, -1.0);
                        }
                        continue;
                    }
                    const double xo = xx + off[0], yo = yy + off[1];
                    const double s = SIFT_SIGMA0 * pow(2.0, (kk + off[2]) / SIFT_S);
                    double angs[SIFT_ORI_BINS], near[SIFT_ORI_BINS], ori_m;
                    int n_near = 0;
                    const int na = orientations_ex(&P->G[o][kk], xo, yo, s, angs, &ori_m, miss ? near : NULL, &n_near, M);
                    for (int a = 0; a < n_near; ++a) add_miss(miss, max_miss, n_miss, o, xo, yo, s, near[a]);
                    const double kp_m = fmin(fmin(fmin((fabs(v) - pre) / pre, ext), fmin(2.0 * half, con_m)),
                                             fmin(edge_m, ori_m));
                    for (int a = 0; a < na; ++a) {
                        if (n == cap) {
                            cap *= 2;
                            all = (kp_full *)realloc(all, sizeof(kp_full) * cap);
                        }
                        kp_full *f = &all[n++];
                        const double scale = ldexp(1.0, o);          /* octave o pixel = 2^o doubled-image pixels */
                        f->kp.x = (xo * scale + 0.5) / 2.0 - 0.5;   /* doubled image -> original (centre-aligned) */
                        f->kp.y = (yo * scale + 0.5) / 2.0 - 0.5;
                        f->kp.sigma = s * scale / 2.0;
                        f->kp.angle = angs[a];
                        f->kp.response = fabs(contrast);
                        f->kp.octave = o;
                        f->kp.layer = kk;
                        f->xo = xo;
                        f->yo = yo;
                        f->s = s;
                        f->o = o;
                        f->k = kk;
                        f->margin = kp_m;
                    }
                }
        }
    qsort(all, n, sizeof(kp_full), kpf_cmp);
    const int m = n < max_kp ? n : max_kp;
    for (int i = 0; i < m; ++i) {
        kps[i] = all[i].kp;
        if (margin) margin[i] = all[i].margin;
        if (desc) descriptor(&P->G[all[i].o][all[i].k], all[i].xo, all[i].yo, all[i].s, all[i].kp.angle,
                             desc + (size_t)128 * i);
    }
    free(all);
    free_pyramid(P);
    free(P);
    return m;
}

/* Step 6: for every query descriptor, the nearest and second-nearest train
 * descriptors by squared L2 distance in fp64 (lowest index on ties); accepted
 * when d1 < ratio^2 d2 (Lowe's ratio test on the distances). */
void oracle_sift_match(const float *q, int nq, const float *t, int nt, double ratio, int32_t *best, double *d1,
                       double *d2, uint8_t *accepted)
{
    for (int i = 0; i < nq; ++i) {
        double b1 = INFINITY, b2 = INFINITY;
        int bi = -1;
        for (int j = 0; j < nt; ++j) {
            double d = 0.0;
            for (int c = 0; c < 128; ++c) {
                const double e = (double)q[(size_t)i * 128 + c] - (double)t[(size_t)j * 128 + c];
                d += e * e;
            }
            if (d < b1) {
                b2 = b1;
                b1 = d;
                bi = j;
            } else if (d < b2) {
                b2 = d;
            }
        }
        best[i] = bi;
        d1[i] = b1;
        d2[i] = b2;
        accepted[i] = (uint8_t)(bi >= 0 && nt >= 2 && b1 < ratio * ratio * b2);
    }
}

int oracle_sizeof_sift_kp(void) { return (int)sizeof(oracle_sift_kp); }

/* Step 6 with the decisions taken in single precision, as the GPU matcher
 * takes them (an argmax decided in floating point is decided in the same
 * precision on both sides).  The squared distance of query i and train j is
 * the fp32 sum over c = 0, 1, ..., 127 in that order of e_c^2, e_c = q_c - t_c
 * rounded to fp32, each term added by one fused multiply-add (d = fma(e_c,
 * e_c, d)), so every implementation that keeps this order gets the same bits.
 * best = the lowest index among the smallest distances, d2 = the second
 * smallest (d2 = d1 on a tie), both INFINITY when there is none; accepted when
 * nt >= 2 and d1 < r2 * d2 in fp32, r2 = (float)(ratio * ratio). */
void oracle_sift_match_f32(const float *q, int nq, const float *t, int nt, double ratio, int32_t *best, float *d1,
                           float *d2, uint8_t *accepted)
{
    const float r2 = (float)(ratio * ratio);
    for (int i = 0; i < nq; ++i) {
        float b1 = INFINITY, b2 = INFINITY;
        int bi = -1;
        for (int j = 0; j < nt; ++j) {
            float d = 0.0f;
            for (int c = 0; c < 128; ++c) {
                const float e = q[(size_t)i * 128 + c] - t[(size_t)j * 128 + c];
                d = fmaf(e, e, d);
            }
            if (d < b1) {
                b2 = b1;
                b1 = d;
                bi = j;
            } else if (d < b2) {
                b2 = d;
            }
        }
        best[i] = bi;
        d1[i] = b1;
        d2[i] = b2;
        accepted[i] = (uint8_t)(bi >= 0 && nt >= 2 && b1 < r2 * b2);
    }
}
