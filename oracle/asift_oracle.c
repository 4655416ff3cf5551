/*
 * asift_oracle.c -- plain, slow, obviously correct CPU oracle for the
 * affine-view-simulation + ORB + brute-force Hamming matching hot path of
 * "Feature Point Extraction for Extra-Affine Image" (arXiv 2503.03479).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package smoke check and the bench's CPU
 * baseline do.  It shares no code, header, table or constant generator with the
 * CUDA path: every table it needs (view table, Gaussian taps, orientation
 * boundaries, steered sampling pattern) is generated here from its written
 * definition.
 *
 * Arithmetic: the warp is fp64 (geometry in exact Q32 fixed point, see
 * oracle_view_table); every ORB and matching step is exact integer arithmetic.
 * Single-threaded, scalar, no SIMD, no blocking or fusion beyond what each
 * definition states.  Compile with -ffp-contract=off so that double results do
 * not depend on the host's FMA contraction.
 *
 * Paper references (section / equation):
 *   Eq. (2)        affine decomposition A = T R1(psi) S T_tau R2(phi)
 *   Sec. III-B     tilt/longitude sampling t = a^k (a = sqrt 2), phi = j b/t, b = 72 deg
 *   Eq. (3), (4)   Lanczos interpolation, L(x;a) = sinc(x) sinc(x/a) on |x| < a
 *   Sec. III-B     ORB (oFAST + rBRIEF) coarse extraction, brute-force Hamming matcher
 *   Sec. IV-C      nearest / second-nearest distance ratio test
 *   Sec. III-B     nearest-neighbour interpolation and scale s of the coarse stage
 *   Eq. (5)-(7)    precision, reprojection threshold, inlier ratio; RANSAC [28] (Sec. III-C)
 *   Sec. III-C     Lanczos reproduction of the best view with n = 4 (8 x 8 window)
 *   Eq. (1)        scaling coefficient of the base-image selection (Sec. III-A)
 * ORB internals the paper does not state (pyramid, FAST-9, Harris, centroid
 * orientation, steered BRIEF) follow the ORB paper cited as [23]; where that is
 * silent, the reading chosen is stated at each function.
 *
 * Pins: every function below is checked by tests/test_oracle_pins.py against
 * closed forms, exact special cases, library routines or brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q31 2147483648.0               /* 2^31 */
#define ORB_BORDER 16                  /* keypoint border, patch radius 15 + 1 */
#define PATCH_R2 225                   /* disc x^2 + y^2 <= 15^2 */
#define N_BINS 30                      /* 12-degree orientation bins */
#define N_PAIRS 256                    /* rBRIEF-256 */

/* ------------------------------------------------------------------------ */
/* trig of an angle in degrees, exact at multiples of 90 degrees             */
/* ------------------------------------------------------------------------ */
static void sincos_deg(double deg, double *s, double *c)
{
    if (fmod(deg, 90.0) == 0.0) {
        long q = ((long)(deg / 90.0) % 4 + 4) % 4;
        static const double S[4] = {0.0, 1.0, 0.0, -1.0};
        static const double C[4] = {1.0, 0.0, -1.0, 0.0};
        *s = S[q];
        *c = C[q];
        return;
    }
    double r = deg * (M_PI / 180.0);
    *s = sin(r);
    *c = cos(r);
}

/* ------------------------------------------------------------------------ */
/* View table (Sec. III-B sampling rule, Eq. (2) with psi = 0, s = 1)        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t k, j;            /* tilt exponent, longitude index                 */
    int32_t W, H;            /* source image size                              */
    int32_t Wr, Hr;          /* rotated canvas size                            */
    int32_t Wv, Hv;          /* view size (Hv == Hr)                           */
    int32_t K;               /* Gaussian half width ceil(4 sigma)              */
    int32_t pad;
    double t, phi_deg, sigma;
    double scale;            /* s of Eq. (2): the canvas magnifies the source by s */
    int64_t cq, sq, tq;      /* round(cos phi / s 2^31), round(sin phi / s 2^31), round(t 2^31) */
} oracle_view;

static double tilt_of(int k)
{
    return (k % 2 == 0) ? ldexp(1.0, k / 2) : ldexp(sqrt(2.0), (k - 1) / 2);
}

/* Fills a view descriptor for a tilt t >= 1 and longitude phi (degrees). */
/*
 * A view with scale: Eq. (2)'s S magnifies the rotated source by `scale`
 * before the tilt, so canvas pixel (i, j) samples
 *   p = R(phi)^T ((i, j) - c_r) / scale + c_s
 * and the canvas is the scaled bounding box of the rotated image.  The
 * Gaussian anti-alias depends on t only.
 */
void oracle_make_view_scaled(int H, int W, double t, double phi, double scale, oracle_view *v)
{
    memset(v, 0, sizeof *v);
    double s, c;
    sincos_deg(phi, &s, &c);
    v->k = -1;
    v->W = W;
    v->H = H;
    v->t = t;
    v->phi_deg = phi;
    v->scale = scale;
    v->Wr = (int32_t)ceil(scale * ((double)W * fabs(c) + (double)H * fabs(s)) - 1e-9);
    v->Hr = (int32_t)ceil(scale * ((double)W * fabs(s) + (double)H * fabs(c)) - 1e-9);
    v->Wv = (int32_t)ceil((double)v->Wr / t);
    v->Hv = v->Hr;
    v->sigma = (t == 1.0) ? 0.0 : 0.8 * sqrt(t * t - 1.0);
    v->K = (int32_t)ceil(4.0 * v->sigma);
    v->cq = llrint(c / scale * Q31);
    v->sq = llrint(s / scale * Q31);
    v->tq = llrint(t * Q31);
}

void oracle_make_view(int H, int W, double t, double phi, oracle_view *v)
{
    oracle_make_view_scaled(H, W, t, phi, 1.0, v);
}

/* View (k, j) of the sampling rule: t = sqrt(2)^k, phi = j 72 / t degrees,
 * scale 1 + k ds. */
static void make_view(int H, int W, int k, int j, double ds, oracle_view *v)
{
    double t = tilt_of(k);
    oracle_make_view_scaled(H, W, t, (k == 0) ? 0.0 : (double)j * 72.0 / t, 1.0 + (double)k * ds, v);
    v->k = k;
    v->j = j;
}

/*
 * Sampling rule of Sec. III-B: t = sqrt(2)^k, k = 0..kmax; for t > 1,
 * phi = j*72/t degrees for every j >= 0 with j*72/t < 180.  At t = 1 a single
 * view (phi = 0) is taken, since every rotation of an untilted image is a
 * similarity that ORB's own orientation already absorbs (the ASIFT convention).
 * Returns the number of views; writes at most cap descriptors.
 */
static int view_table_ds(int H, int W, int kmax, double ds, oracle_view *out, int cap)
{
    int n = 0;
    for (int k = 0; k <= kmax; ++k) {
        double t = tilt_of(k);
        for (int j = 0;; ++j) {
            if (k == 0 && j > 0) break;
            if (k > 0 && !((double)j * 72.0 / t < 180.0)) break;
            if (n < cap) make_view(H, W, k, j, ds, &out[n]);
            ++n;
        }
    }
    return n;
}

int oracle_view_table(int H, int W, int kmax, oracle_view *out, int cap)
{
    return view_table_ds(H, W, kmax, 0.0, out, cap);
}

/*
 * The coarse stage's parameter groups (Sec. III-B): the same (t, phi) list
 * with the scale s = 1 + k ds tied to the tilt exponent k (the paper takes
 * ds = 0.5 and n = 5, so s runs 1, 1.5, ..., 3.5).
 */
int oracle_view_table_scaled(int H, int W, int kmax, double ds, oracle_view *out, int cap)
{
    return view_table_ds(H, W, kmax, ds, out, cap);
}

/* Gaussian taps g_0..g_K along the tilt axis, g_k ~ exp(-k^2 / 2 sigma^2),
 * normalised so that g_0 + 2 sum_{k>=1} g_k = 1.  sigma = 0 gives g_0 = 1. */
void oracle_gauss_taps(double sigma, int K, double *g)
{
    if (K == 0 || sigma == 0.0) {
        g[0] = 1.0;
        return;
    }
    double sum = 0.0;
    for (int k = 0; k <= K; ++k) {
        g[k] = exp(-(double)k * (double)k / (2.0 * sigma * sigma));
        sum += (k == 0) ? g[k] : 2.0 * g[k];
    }
    for (int k = 0; k <= K; ++k) g[k] /= sum;
}

/* ------------------------------------------------------------------------ */
/* Lanczos-3 kernel, Eq. (4), and normalised 6-tap weights, Eq. (3)          */
/* ------------------------------------------------------------------------ */
/* sinc(x) = sin(pi x)/(pi x), sinc(0) = 1, and exactly 0 at the other integers
 * (where the double sin(pi x) would leave a rounding residue). */
static double sinc(double x)
{
    if (x == 0.0) return 1.0;
    if (x == floor(x)) return 0.0;
    double px = M_PI * x;
    return sin(px) / px;
}

/* L(x; 3) = sinc(x) sinc(x/3) for |x| < 3, else 0 (Eq. (4) with a = 3). */
double oracle_lanczos3(double x)
{
    if (!(fabs(x) < 3.0)) return 0.0;
    return sinc(x) * sinc(x / 3.0);
}

/* Weights for taps floor(p) + m, m = -2..3, at fractional part f in [0,1):
 * w_m = L(f - m) / sum_m' L(f - m').  Eq. (3) with its garbled limits read as
 * i = -a+1 .. a (2a = 6 taps); the weights are normalised so they sum to 1. */
void oracle_lanczos3_weights(double f, double w[6])
{
    double sum = 0.0;
    for (int m = -2; m <= 3; ++m) {
        w[m + 2] = oracle_lanczos3(f - (double)m);
        sum += w[m + 2];
    }
    for (int i = 0; i < 6; ++i) w[i] /= sum;
}

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Q32 fixed-point source coordinate of canvas pixel (i, jrow):
 * p = R(phi)^T ((i, j) - c_r) + c_s with c = (size - 1)/2 per axis. */
static void canvas_to_src(const oracle_view *v, int i, int jrow, int64_t *px, int64_t *py)
{
    int64_t dx2 = 2 * (int64_t)i - v->Wr + 1;     /* 2 (i - c_rx) */
    int64_t dy2 = 2 * (int64_t)jrow - v->Hr + 1;  /* 2 (j - c_ry) */
    *px = v->cq * dx2 + v->sq * dy2 + (int64_t)(v->W - 1) * (int64_t)2147483648LL;
    *py = -v->sq * dx2 + v->cq * dy2 + (int64_t)(v->H - 1) * (int64_t)2147483648LL;
}

static inline double q32_frac(int64_t q) { return (double)(uint32_t)(q & 0xffffffffLL) / 4294967296.0; }
static inline int64_t q32_floor(int64_t q) { return q >> 32; }   /* arithmetic shift = floor */

/* Canvas value C(i, j): Lanczos-3 sample of u at p (Eq. (3)), clamp-to-edge
 * taps; 0 where p lies outside [-0.5, W-0.5) x [-0.5, H-0.5). */
static double canvas_value(const double *u, int pitch, const oracle_view *v, int i, int jrow)
{
    int64_t px, py;
    canvas_to_src(v, i, jrow, &px, &py);
    const int64_t half = 2147483648LL;
    if (px < -half || px >= (int64_t)(2 * v->W - 1) * half) return 0.0;
    if (py < -half || py >= (int64_t)(2 * v->H - 1) * half) return 0.0;
    int x0 = (int)q32_floor(px), y0 = (int)q32_floor(py);
    double wx[6], wy[6];
    oracle_lanczos3_weights(q32_frac(px), wx);
    oracle_lanczos3_weights(q32_frac(py), wy);
    double acc = 0.0;
    for (int n = -2; n <= 3; ++n) {
        int yy = clampi(y0 + n, 0, v->H - 1);
        double row = 0.0;
        for (int m = -2; m <= 3; ++m) {
            int xx = clampi(x0 + m, 0, v->W - 1);
            row += wx[m + 2] * u[(size_t)yy * pitch + xx];
        }
        acc += wy[n + 2] * row;
    }
    return acc;
}

/* Canvas validity for the mask: p inside the footprint shrunk by one pixel,
 * [0.5, W-1.5] x [0.5, H-1.5]; canvas columns outside [0, Wr) are invalid. */
static int canvas_valid(const oracle_view *v, int i, int jrow)
{
    if (i < 0 || i >= v->Wr) return 0;
    int64_t px, py;
    canvas_to_src(v, i, jrow, &px, &py);
    const int64_t half = 2147483648LL;
    return px >= half && px <= (int64_t)(2 * v->W - 3) * half &&
           py >= half && py <= (int64_t)(2 * v->H - 3) * half;
}

/*
 * One simulated view (Eq. (2) with psi = 0, s = 1, translation 0):
 *   C = Lanczos-3 rotation of u by phi into the Wr x Hr canvas   (Eq. (3)-(4))
 *   B = 1-D Gaussian (sigma = 0.8 sqrt(t^2-1)) along canvas x, clamped rows
 *   v(x', j) = Lanczos-3 sample of B's row j at canvas x = t (x' - (Wv-1)/2) + (Wr-1)/2,
 *              the tilt T_tau compressing x by t (position in Q32 fixed point)
 *   v_u8 = clamp(rint(v), 0, 255) (ties to even), mask = both canvas
 *   neighbours of x valid.
 * Any output pointer may be NULL.  Output rows have pitch Wv.
 */
void oracle_warp_view_f64(const double *u, int pitch, const oracle_view *v,
                          double *out_f64, uint8_t *out_u8, uint8_t *out_mask)
{
    const int Wr = v->Wr, Hr = v->Hr, Wv = v->Wv, K = v->K;
    double g[128];
    oracle_gauss_taps(v->sigma, K, g);
    double *C = (double *)malloc(sizeof(double) * (size_t)Wr);
    double *B = (double *)malloc(sizeof(double) * (size_t)Wr);
    for (int j = 0; j < Hr; ++j) {
        for (int i = 0; i < Wr; ++i) C[i] = canvas_value(u, pitch, v, i, j);
        for (int i = 0; i < Wr; ++i) {
            double acc = 0.0;
            for (int k = -K; k <= K; ++k) acc += g[abs(k)] * C[clampi(i - k, 0, Wr - 1)];
            B[i] = acc;
        }
        for (int x = 0; x < Wv; ++x) {
            int64_t X = v->tq * (2 * (int64_t)x - Wv + 1) + (int64_t)(Wr - 1) * (int64_t)2147483648LL;
            int x0 = (int)q32_floor(X);
            double w[6];
            oracle_lanczos3_weights(q32_frac(X), w);
            double acc = 0.0;
            for (int m = -2; m <= 3; ++m) acc += w[m + 2] * B[clampi(x0 + m, 0, Wr - 1)];
            size_t o = (size_t)j * Wv + x;
            if (out_f64) out_f64[o] = acc;
            if (out_u8) {
                double r = nearbyint(acc);
                out_u8[o] = (uint8_t)(r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r));
            }
            if (out_mask) out_mask[o] = (uint8_t)(canvas_valid(v, x0, j) && canvas_valid(v, x0 + 1, j));
        }
    }
    free(C);
    free(B);
}

/* The same view of an 8-bit source image. */
void oracle_warp_view(const uint8_t *u, int pitch, const oracle_view *v,
                      double *out_f64, uint8_t *out_u8, uint8_t *out_mask)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)v->W * v->H);
    for (int y = 0; y < v->H; ++y)
        for (int x = 0; x < v->W; ++x) d[(size_t)y * v->W + x] = (double)u[(size_t)y * pitch + x];
    oracle_warp_view_f64(d, v->W, v, out_f64, out_u8, out_mask);
    free(d);
}

/* Nearest-neighbour form of the view, the interpolation the coarse stage
 * uses (Sec. III-B): the Lanczos-3 samples of the rotation and of the tilt
 * become the value of the nearest pixel, round(p) = floor(p + 1/2) taken in
 * Q32, with the same background rule (0 outside [-0.5, W-0.5) x
 * [-0.5, H-0.5)), the same Gaussian along canvas x before the tilt, the same
 * quantisation and the same mask.  The tilt's nearest canvas column is
 * clamped to [0, Wr-1]. */
static double canvas_value_nn(const double *u, int pitch, const oracle_view *v, int i, int jrow)
{
    int64_t px, py;
    canvas_to_src(v, i, jrow, &px, &py);
    const int64_t half = 2147483648LL;
    if (px < -half || px >= (int64_t)(2 * v->W - 1) * half) return 0.0;
    if (py < -half || py >= (int64_t)(2 * v->H - 1) * half) return 0.0;
    const int xs = (int)q32_floor(px + half), ys = (int)q32_floor(py + half);
    return u[(size_t)ys * pitch + xs];
}

void oracle_warp_view_nn_f64(const double *u, int pitch, const oracle_view *v,
                             double *out_f64, uint8_t *out_u8, uint8_t *out_mask)
{
    const int Wr = v->Wr, Hr = v->Hr, Wv = v->Wv, K = v->K;
    const int64_t half = 2147483648LL;
    double g[128];
    oracle_gauss_taps(v->sigma, K, g);
    double *Crow = (double *)malloc(sizeof(double) * (size_t)Wr);
    for (int j = 0; j < Hr; ++j) {
        for (int i = 0; i < Wr; ++i) Crow[i] = canvas_value_nn(u, pitch, v, i, j);
        for (int x = 0; x < Wv; ++x) {
            int64_t X = v->tq * (2 * (int64_t)x - Wv + 1) + (int64_t)(Wr - 1) * half;
            const int xn = clampi((int)q32_floor(X + half), 0, Wr - 1);
            /* B(xn) = sum_k g_|k| C(clamp(xn - k)) */
            double acc = 0.0;
            for (int k = -K; k <= K; ++k) acc += g[abs(k)] * Crow[clampi(xn - k, 0, Wr - 1)];
            const int x0 = (int)q32_floor(X);
            size_t o = (size_t)j * Wv + x;
            if (out_f64) out_f64[o] = acc;
            if (out_u8) {
                double r = nearbyint(acc);
                out_u8[o] = (uint8_t)(r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r));
            }
            if (out_mask) out_mask[o] = (uint8_t)(canvas_valid(v, x0, j) && canvas_valid(v, x0 + 1, j));
        }
    }
    free(Crow);
}

void oracle_warp_view_nn(const uint8_t *u, int pitch, const oracle_view *v,
                         double *out_f64, uint8_t *out_u8, uint8_t *out_mask)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)v->W * v->H);
    for (int y = 0; y < v->H; ++y)
        for (int x = 0; x < v->W; ++x) d[(size_t)y * v->W + x] = (double)u[(size_t)y * pitch + x];
    oracle_warp_view_nn_f64(d, v->W, v, out_f64, out_u8, out_mask);
    free(d);
}

/* Lanczos-a views for the precise stage's reproduction of the best view
 * (Sec. III-C: Lanczos with n = 4, an 8 x 8 window): Eq. (3)-(4) with a
 * general a, otherwise the view of oracle_warp_view_f64 (same geometry,
 * background, Gaussian, quantisation and mask). */
double oracle_lanczos(double x, int a)
{
    if (!(fabs(x) < (double)a)) return 0.0;
    return sinc(x) * sinc(x / (double)a);
}

/* Normalised weights of taps floor(p) + m, m = -a+1 .. a (2a taps), at
 * fractional part f in [0, 1). */
void oracle_lanczos_weights(double f, int a, double *w)
{
    double sum = 0.0;
    for (int m = -a + 1; m <= a; ++m) {
        w[m + a - 1] = oracle_lanczos(f - (double)m, a);
        sum += w[m + a - 1];
    }
    for (int i = 0; i < 2 * a; ++i) w[i] /= sum;
}

static double canvas_value_a(const double *u, int pitch, const oracle_view *v, int i, int jrow, int a)
{
    int64_t px, py;
    canvas_to_src(v, i, jrow, &px, &py);
    const int64_t half = 2147483648LL;
    if (px < -half || px >= (int64_t)(2 * v->W - 1) * half) return 0.0;
    if (py < -half || py >= (int64_t)(2 * v->H - 1) * half) return 0.0;
    int x0 = (int)q32_floor(px), y0 = (int)q32_floor(py);
    double wx[16], wy[16];
    oracle_lanczos_weights(q32_frac(px), a, wx);
    oracle_lanczos_weights(q32_frac(py), a, wy);
    double acc = 0.0;
    for (int n = -a + 1; n <= a; ++n) {
        int yy = clampi(y0 + n, 0, v->H - 1);
        double row = 0.0;
        for (int m = -a + 1; m <= a; ++m) {
            int xx = clampi(x0 + m, 0, v->W - 1);
            row += wx[m + a - 1] * u[(size_t)yy * pitch + xx];
        }
        acc += wy[n + a - 1] * row;
    }
    return acc;
}

/* a in [1, 8]. */
void oracle_warp_view_lanczos_f64(const double *u, int pitch, const oracle_view *v, int a,
                                  double *out_f64, uint8_t *out_u8, uint8_t *out_mask)
{
    const int Wr = v->Wr, Hr = v->Hr, Wv = v->Wv, K = v->K;
    double g[128];
    oracle_gauss_taps(v->sigma, K, g);
    double *Crow = (double *)malloc(sizeof(double) * (size_t)Wr);
    double *B = (double *)malloc(sizeof(double) * (size_t)Wr);
    for (int j = 0; j < Hr; ++j) {
        for (int i = 0; i < Wr; ++i) Crow[i] = canvas_value_a(u, pitch, v, i, j, a);
        for (int i = 0; i < Wr; ++i) {
            double acc = 0.0;
            for (int k = -K; k <= K; ++k) acc += g[abs(k)] * Crow[clampi(i - k, 0, Wr - 1)];
            B[i] = acc;
        }
        for (int x = 0; x < Wv; ++x) {
            int64_t X = v->tq * (2 * (int64_t)x - Wv + 1) + (int64_t)(Wr - 1) * (int64_t)2147483648LL;
            int x0 = (int)q32_floor(X);
            double w[16];
            oracle_lanczos_weights(q32_frac(X), a, w);
            double acc = 0.0;
            for (int m = -a + 1; m <= a; ++m) acc += w[m + a - 1] * B[clampi(x0 + m, 0, Wr - 1)];
            size_t o = (size_t)j * Wv + x;
            if (out_f64) out_f64[o] = acc;
            if (out_u8) {
                double r = nearbyint(acc);
                out_u8[o] = (uint8_t)(r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r));
            }
            if (out_mask) out_mask[o] = (uint8_t)(canvas_valid(v, x0, j) && canvas_valid(v, x0 + 1, j));
        }
    }
    free(Crow);
    free(B);
}

void oracle_warp_view_lanczos(const uint8_t *u, int pitch, const oracle_view *v, int a,
                              double *out_f64, uint8_t *out_u8, uint8_t *out_mask)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)v->W * v->H);
    for (int y = 0; y < v->H; ++y)
        for (int x = 0; x < v->W; ++x) d[(size_t)y * v->W + x] = (double)u[(size_t)y * pitch + x];
    oracle_warp_view_lanczos_f64(d, v->W, v, a, out_f64, out_u8, out_mask);
    free(d);
}

/* ------------------------------------------------------------------------ */
/* ORB scale pyramid (scale factor 1.2)                                      */
/* ------------------------------------------------------------------------ */
/* W_l = round-half-up(W_0 (5/6)^l), evaluated exactly in integers. */
int oracle_level_size(int n0, int l)
{
    int64_t p5 = 1, p6 = 1;
    for (int i = 0; i < l; ++i) { p5 *= 5; p6 *= 6; }
    return (int)((2 * (int64_t)n0 * p5 + p6) / (2 * p6));
}

/* Level l (size Wl x Hl) from level l-1 (Wp x Hp) by centre-aligned bilinear
 * interpolation in exact integers: source x = ((2x+1) Wp - Wl) / (2 Wl),
 * weights in Q11, result rounded half up; the mask needs all four taps valid. */
void oracle_downscale(const uint8_t *src, const uint8_t *msrc, int Wp, int Hp,
                      uint8_t *dst, uint8_t *mdst, int Wl, int Hl)
{
    for (int y = 0; y < Hl; ++y) {
        int64_t ny = (2 * (int64_t)y + 1) * Hp - Hl, dy = 2 * (int64_t)Hl;
        int y0 = (int)(ny / dy);
        int fy = (int)(((ny - y0 * dy) << 11) / dy);
        int y1 = y0 + 1 < Hp ? y0 + 1 : Hp - 1;
        for (int x = 0; x < Wl; ++x) {
            int64_t nx = (2 * (int64_t)x + 1) * Wp - Wl, dx = 2 * (int64_t)Wl;
            int x0 = (int)(nx / dx);
            int fx = (int)(((nx - x0 * dx) << 11) / dx);
            int x1 = x0 + 1 < Wp ? x0 + 1 : Wp - 1;
            int64_t a = src[(size_t)y0 * Wp + x0], b = src[(size_t)y0 * Wp + x1];
            int64_t c = src[(size_t)y1 * Wp + x0], d = src[(size_t)y1 * Wp + x1];
            int64_t s = (int64_t)(2048 - fx) * (2048 - fy) * a + (int64_t)fx * (2048 - fy) * b +
                        (int64_t)(2048 - fx) * fy * c + (int64_t)fx * fy * d;
            dst[(size_t)y * Wl + x] = (uint8_t)((s + (1 << 21)) >> 22);
            if (mdst)
                mdst[(size_t)y * Wl + x] = (uint8_t)(msrc[(size_t)y0 * Wp + x0] && msrc[(size_t)y0 * Wp + x1] &&
                                                    msrc[(size_t)y1 * Wp + x0] && msrc[(size_t)y1 * Wp + x1]);
        }
    }
}

/* Smoothing for the BRIEF tests: separable 7-tap integer binomial-like kernel
 * [18 34 49 54 49 34 18] / 256 per axis (about sigma = 2, as ORB [23] smooths
 * before its tests), clamp-to-edge; horizontal sum kept exactly, the final
 * 2-D sum rounded half up by 2^16. */
static const int SMOOTH7[7] = {18, 34, 49, 54, 49, 34, 18};

void oracle_smooth(const uint8_t *src, int W, int H, uint8_t *dst)
{
    uint32_t *h = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)W * H);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint32_t s = 0;
            for (int i = 0; i < 7; ++i) s += (uint32_t)SMOOTH7[i] * src[(size_t)y * W + clampi(x + i - 3, 0, W - 1)];
            h[(size_t)y * W + x] = s;
        }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint32_t s = 0;
            for (int i = 0; i < 7; ++i) s += (uint32_t)SMOOTH7[i] * h[(size_t)clampi(y + i - 3, 0, H - 1) * W + x];
            dst[(size_t)y * W + x] = (uint8_t)((s + 32768u) >> 16);
        }
    free(h);
}

/* ------------------------------------------------------------------------ */
/* FAST-9 (Rosten & Drummond, as used by ORB [23])                           */
/* ------------------------------------------------------------------------ */
/* Bresenham circle of radius 3: 16 offsets from (0,-3), clockwise on screen. */
static const int CIRC[16][2] = {{0, -3}, {1, -3}, {2, -2}, {3, -1}, {3, 0}, {3, 1}, {2, 2}, {1, 3},
                                {0, 3}, {-1, 3}, {-2, 2}, {-3, 1}, {-3, 0}, {-3, -1}, {-2, -2}, {-1, -3}};

/* 1 iff some 9 cyclically consecutive circle pixels are all > I_p + thr, or all
 * < I_p - thr (strict).  The caller keeps (x, y) at least 3 px inside. */
int oracle_fast9(const uint8_t *img, int W, int x, int y, int thr)
{
    int c = img[(size_t)y * W + x];
    for (int start = 0; start < 16; ++start) {
        int all_b = 1, all_d = 1;
        for (int i = 0; i < 9; ++i) {
            const int *o = CIRC[(start + i) & 15];
            int v = img[(size_t)(y + o[1]) * W + x + o[0]];
            if (!(v > c + thr)) all_b = 0;
            if (!(v < c - thr)) all_d = 0;
        }
        if (all_b || all_d) return 1;
    }
    return 0;
}

/* Harris response scaled by 25: R25 = 25 (a b - c^2) - (a + b)^2 with
 * a = sum Ix^2, b = sum Iy^2, c = sum Ix Iy over the 7x7 window centred at
 * (x, y), Ix / Iy the 3x3 Sobel derivatives.  Equals 25 (det - 0.04 tr^2)
 * exactly (k = 0.04 = 1/25).  The caller keeps (x, y) at least 4 px inside. */
int64_t oracle_harris25(const uint8_t *img, int W, int x, int y)
{
    int64_t a = 0, b = 0, c = 0;
    for (int dy = -3; dy <= 3; ++dy)
        for (int dx = -3; dx <= 3; ++dx) {
            int X = x + dx, Y = y + dy;
#define P(xx, yy) ((int64_t)img[(size_t)(yy) * W + (xx)])
            int64_t ix = (P(X + 1, Y - 1) + 2 * P(X + 1, Y) + P(X + 1, Y + 1)) -
                         (P(X - 1, Y - 1) + 2 * P(X - 1, Y) + P(X - 1, Y + 1));
            int64_t iy = (P(X - 1, Y + 1) + 2 * P(X, Y + 1) + P(X + 1, Y + 1)) -
                         (P(X - 1, Y - 1) + 2 * P(X, Y - 1) + P(X + 1, Y - 1));
#undef P
            a += ix * ix;
            b += iy * iy;
            c += ix * iy;
        }
    return 25 * (a * b - c * c) - (a + b) * (a + b);
}

/* A corner candidate: inside the border, the four corners of its 33x33 box
 * mask-valid, and FAST-9 positive. */
static int is_corner(const uint8_t *img, const uint8_t *mask, int W, int H, int x, int y, int thr)
{
    if (x < ORB_BORDER || x >= W - ORB_BORDER || y < ORB_BORDER || y >= H - ORB_BORDER) return 0;
    const int b = ORB_BORDER;
    if (!(mask[(size_t)(y - b) * W + x - b] && mask[(size_t)(y - b) * W + x + b] &&
          mask[(size_t)(y + b) * W + x - b] && mask[(size_t)(y + b) * W + x + b]))
        return 0;
    return oracle_fast9(img, W, x, y, thr);
}

typedef struct {
    int32_t x, y;
    int64_t r;
} cand;

/* Order: Harris response descending, then y ascending, then x ascending. */
static int cand_cmp(const void *pa, const void *pb)
{
    const cand *a = (const cand *)pa, *b = (const cand *)pb;
    if (a->r != b->r) return a->r > b->r ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    return 0;
}

/*
 * FAST + Harris + 3x3 non-maximum suppression on one level.  A corner p
 * survives iff for every corner n among its 8 neighbours, R(p) > R(n) or
 * (R(p) == R(n) and p precedes n in raster order).  Writes the survivors
 * (unsorted, raster order) and returns their count (may exceed cap; only cap
 * are written).
 */
int oracle_detect_level(const uint8_t *img, const uint8_t *mask, int W, int H, int thr,
                        int32_t *xs, int32_t *ys, int64_t *rs, int cap)
{
    uint8_t *isc = (uint8_t *)calloc((size_t)W * H, 1);
    int64_t *R = (int64_t *)calloc((size_t)W * H, sizeof(int64_t));
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            if (is_corner(img, mask, W, H, x, y, thr)) {
                isc[(size_t)y * W + x] = 1;
                R[(size_t)y * W + x] = oracle_harris25(img, W, x, y);
            }
    int n = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            if (!isc[p]) continue;
            int keep = 1;
            for (int dy = -1; dy <= 1 && keep; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy) continue;
                    size_t q = (size_t)(y + dy) * W + (x + dx);
                    if (!isc[q]) continue;
                    if (!(R[p] > R[q] || (R[p] == R[q] && p < q))) { keep = 0; break; }
                }
            if (keep) {
                if (n < cap) { xs[n] = x; ys[n] = y; rs[n] = R[p]; }
                ++n;
            }
        }
    free(isc);
    free(R);
    return n;
}

/* Per-level keypoint quota: q_l = floor(N A_l / sum A), remainder to level 0. */
void oracle_quota(const int *Ws, const int *Hs, int L, int N, int *q)
{
    int64_t S = 0, used = 0;
    for (int l = 0; l < L; ++l) S += (int64_t)Ws[l] * Hs[l];
    for (int l = 0; l < L; ++l) {
        q[l] = (int)((int64_t)N * Ws[l] * Hs[l] / S);
        used += q[l];
    }
    q[0] += (int)(N - used);
}

/* ------------------------------------------------------------------------ */
/* Orientation (intensity centroid, ORB [23]) and steered rBRIEF             */
/* ------------------------------------------------------------------------ */
/* Boundary unit vectors of the 30 sectors, Q30: e_b at angle b*12 - 6 degrees
 * for b < 15, e_{b+15} = -e_b. */
void oracle_bin_table(int64_t e[N_BINS][2])
{
    for (int b = 0; b < 15; ++b) {
        double s, c;
        sincos_deg((double)b * 12.0 - 6.0, &s, &c);
        e[b][0] = llrint(c * 1073741824.0);
        e[b][1] = llrint(s * 1073741824.0);
        e[b + 15][0] = -e[b][0];
        e[b + 15][1] = -e[b][1];
    }
}

/* Sector of (mx, my): the b with (mx,my) on or left of e_b and strictly right
 * of e_{b+1}, i.e. angle in [(b - 0.5) 12, (b + 0.5) 12) degrees.  (0,0) -> 0. */
int oracle_angle_bin(int64_t mx, int64_t my)
{
    if (mx == 0 && my == 0) return 0;
    int64_t e[N_BINS][2];
    oracle_bin_table(e);
    for (int b = 0; b < N_BINS; ++b) {
        const int64_t *lo = e[b], *hi = e[(b + 1) % N_BINS];
        int64_t c0 = lo[0] * my - lo[1] * mx;
        int64_t c1 = hi[0] * my - hi[1] * mx;
        if (c0 >= 0 && c1 < 0) return b;
    }
    return -1; /* unreachable for a consistent table */
}

/* Intensity-centroid moments over the disc x^2 + y^2 <= 225 around (x, y). */
void oracle_moments(const uint8_t *img, int W, int x, int y, int64_t *m10, int64_t *m01)
{
    int64_t a = 0, b = 0;
    for (int dy = -15; dy <= 15; ++dy)
        for (int dx = -15; dx <= 15; ++dx) {
            if (dx * dx + dy * dy > PATCH_R2) continue;
            int64_t v = img[(size_t)(y + dy) * W + x + dx];
            a += dx * v;
            b += dy * v;
        }
    *m10 = a;
    *m01 = b;
}

/* SplitMix64 (Steele, Lea, Flood 2014; constants as published). */
static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * Seeded rBRIEF-256 sampling pattern and its 30 steered copies,
 * pat[b][i] = {px, py, qx, qy} (int8).  Unsteered points: x, y ~ N(0, (31/5)^2)
 * by Box-Muller on SplitMix64 uniforms u = ((z >> 11) + 1) 2^-53, rounded
 * ties-to-even; points outside the radius-15 disc are redrawn, pairs with
 * p == q are redrawn.  Steered copy b < 15: rotation by b*12 degrees, each
 * coordinate rounded half away from zero; copy b + 15 = -(copy b).
 */
void oracle_pattern(uint64_t seed, int8_t pat[N_BINS][N_PAIRS][4])
{
    uint64_t st = seed;
    int base[N_PAIRS][4];
    const double sd = 31.0 / 5.0;
    for (int i = 0; i < N_PAIRS;) {
        int pt[2][2];
        for (int k = 0; k < 2;) {
            double u1 = (double)((splitmix64(&st) >> 11) + 1) * 0x1.0p-53;
            double u2 = (double)((splitmix64(&st) >> 11) + 1) * 0x1.0p-53;
            double r = sqrt(-2.0 * log(u1));
            double a = 2.0 * M_PI * u2;
            int x = (int)nearbyint(sd * r * cos(a));
            int y = (int)nearbyint(sd * r * sin(a));
            if (x * x + y * y > PATCH_R2) continue;
            pt[k][0] = x;
            pt[k][1] = y;
            ++k;
        }
        if (pt[0][0] == pt[1][0] && pt[0][1] == pt[1][1]) continue;
        base[i][0] = pt[0][0];
        base[i][1] = pt[0][1];
        base[i][2] = pt[1][0];
        base[i][3] = pt[1][1];
        ++i;
    }
    for (int b = 0; b < 15; ++b) {
        double s, c;
        sincos_deg((double)b * 12.0, &s, &c);
        for (int i = 0; i < N_PAIRS; ++i)
            for (int k = 0; k < 2; ++k) {
                double x = base[i][2 * k], y = base[i][2 * k + 1];
                int rx = (int)round(c * x - s * y);
                int ry = (int)round(s * x + c * y);
                pat[b][i][2 * k] = (int8_t)rx;
                pat[b][i][2 * k + 1] = (int8_t)ry;
                pat[b + 15][i][2 * k] = (int8_t)(-rx);
                pat[b + 15][i][2 * k + 1] = (int8_t)(-ry);
            }
    }
}

/* Steered BRIEF: bit i = [S(kp + p'_i) < S(kp + q'_i)] on the smoothed level,
 * packed LSB first: bit i in byte i >> 3, position i & 7. */
void oracle_brief(const uint8_t *smooth, int W, int x, int y, int bin,
                  const int8_t pat[N_BINS][N_PAIRS][4], uint8_t desc[32])
{
    memset(desc, 0, 32);
    for (int i = 0; i < N_PAIRS; ++i) {
        const int8_t *p = pat[bin][i];
        int a = smooth[(size_t)(y + p[1]) * W + x + p[0]];
        int b = smooth[(size_t)(y + p[3]) * W + x + p[2]];
        if (a < b) desc[i >> 3] |= (uint8_t)(1u << (i & 7));
    }
}

/* ------------------------------------------------------------------------ */
/* ORB on one view                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int16_t x, y;       /* position in its level */
    uint8_t level, bin; /* pyramid level, orientation bin (angle = 12 bin deg) */
    int16_t pad;
    int64_t r25;        /* Harris response x 25 */
} oracle_kp;

/*
 * ORB on one view: L-level pyramid (scale 1.2), FAST-9 (threshold thr) +
 * Harris + NMS per level, per-level quota of the N keypoints (top by
 * (R25 desc, y, x)), orientation bin from the centroid, steered BRIEF on the
 * smoothed level.  Output order: level ascending, then the selection order.
 * Returns the number of keypoints (<= N).  cand_cap bounds the per-level
 * candidate list; a level with more survivors returns -1 - level.
 */
int oracle_orb_view(const uint8_t *view, const uint8_t *mask, int Wv, int Hv, int L, int N, int thr,
                    const int8_t pat[N_BINS][N_PAIRS][4], oracle_kp *kps, uint8_t (*desc)[32], int cand_cap)
{
    int Ws[16], Hs[16], q[16];
    for (int l = 0; l < L; ++l) {
        Ws[l] = oracle_level_size(Wv, l);
        Hs[l] = oracle_level_size(Hv, l);
    }
    oracle_quota(Ws, Hs, L, N, q);
    uint8_t *img = (uint8_t *)malloc((size_t)Wv * Hv), *msk = (uint8_t *)malloc((size_t)Wv * Hv);
    uint8_t *nimg = (uint8_t *)malloc((size_t)Wv * Hv), *nmsk = (uint8_t *)malloc((size_t)Wv * Hv);
    uint8_t *sm = (uint8_t *)malloc((size_t)Wv * Hv);
    memcpy(img, view, (size_t)Wv * Hv);
    memcpy(msk, mask, (size_t)Wv * Hv);
    cand *cs = (cand *)malloc(sizeof(cand) * (size_t)cand_cap);
    int32_t *xs = (int32_t *)malloc(sizeof(int32_t) * (size_t)cand_cap);
    int32_t *ys = (int32_t *)malloc(sizeof(int32_t) * (size_t)cand_cap);
    int64_t *rs = (int64_t *)malloc(sizeof(int64_t) * (size_t)cand_cap);
    int out = 0, err = 0;
    for (int l = 0; l < L; ++l) {
        int W = Ws[l], H = Hs[l];
        if (l > 0) {
            oracle_downscale(img, msk, Ws[l - 1], Hs[l - 1], nimg, nmsk, W, H);
            memcpy(img, nimg, (size_t)W * H);
            memcpy(msk, nmsk, (size_t)W * H);
        }
        int n = oracle_detect_level(img, msk, W, H, thr, xs, ys, rs, cand_cap);
        if (n > cand_cap) { err = -1 - l; break; }
        for (int i = 0; i < n; ++i) { cs[i].x = xs[i]; cs[i].y = ys[i]; cs[i].r = rs[i]; }
        qsort(cs, (size_t)n, sizeof(cand), cand_cmp);
        int take = n < q[l] ? n : q[l];
        oracle_smooth(img, W, H, sm);
        for (int i = 0; i < take; ++i) {
            int64_t m10, m01;
            oracle_moments(img, W, cs[i].x, cs[i].y, &m10, &m01);
            int bin = oracle_angle_bin(m10, m01);
            oracle_kp *k = &kps[out];
            memset(k, 0, sizeof *k);
            k->x = (int16_t)cs[i].x;
            k->y = (int16_t)cs[i].y;
            k->level = (uint8_t)l;
            k->bin = (uint8_t)bin;
            k->r25 = cs[i].r;
            oracle_brief(sm, W, cs[i].x, cs[i].y, bin, pat, desc[out]);
            ++out;
        }
    }
    free(img); free(msk); free(nimg); free(nmsk); free(sm);
    free(cs); free(xs); free(ys); free(rs);
    return err ? err : out;
}

/* ------------------------------------------------------------------------ */
/* Brute-force Hamming matching with the ratio test                          */
/* ------------------------------------------------------------------------ */
static int hamming256(const uint8_t *a, const uint8_t *b)
{
    int d = 0;
    for (int i = 0; i < 4; ++i) {
        uint64_t x, y;
        memcpy(&x, a + 8 * i, 8);
        memcpy(&y, b + 8 * i, 8);
        d += __builtin_popcountll(x ^ y);
    }
    return d;
}

/*
 * For every query: best = argmin_r H(q, r) (lowest index on ties),
 * d1 = H(q, best), d2 = min_{r != best} H(q, r) (257 if nt < 2);
 * accepted iff nt >= 2 and den * d1 < num * d2 (nearest / second-nearest
 * ratio test with ratio num/den, Sec. IV-C; exact in integers).
 * Returns the number of accepted queries.
 */
int oracle_match(const uint8_t (*q)[32], int nq, const uint8_t (*t)[32], int nt, int num, int den,
                 int32_t *best, int32_t *d1, int32_t *d2, uint8_t *acc)
{
    int n_acc = 0;
    for (int i = 0; i < nq; ++i) {
        int b = -1, bd = 257, sd = 257;
        for (int r = 0; r < nt; ++r) {
            int d = hamming256(q[i], t[r]);
            if (d < bd) { sd = bd; bd = d; b = r; }
            else if (d < sd) sd = d;
        }
        best[i] = b;
        d1[i] = bd;
        d2[i] = sd;
        acc[i] = (uint8_t)(nt >= 2 && (int64_t)den * bd < (int64_t)num * sd);
        n_acc += acc[i];
    }
    return n_acc;
}

/* Back-projection of a keypoint at (xl, yl) of pyramid level l of a view to the
 * source image: level -> level 0 (centre-aligned scale W_0/W_l), -> canvas
 * (x = t (x0 - (Wv-1)/2) + (Wr-1)/2), -> source p = R^T (canvas - c_r) / s + c_s. */
void oracle_backproject(const oracle_view *v, int l, double xl, double yl, double *sx, double *sy)
{
    int W0 = v->Wv, H0 = v->Hv;
    int Wl = oracle_level_size(W0, l), Hl = oracle_level_size(H0, l);
    double x0 = (xl + 0.5) * (double)W0 / (double)Wl - 0.5;
    double y0 = (yl + 0.5) * (double)H0 / (double)Hl - 0.5;
    double X = v->t * (x0 - (v->Wv - 1) * 0.5) + (v->Wr - 1) * 0.5;
    double dx = X - (v->Wr - 1) * 0.5, dy = y0 - (v->Hr - 1) * 0.5;
    double s, c;
    sincos_deg(v->phi_deg, &s, &c);
    const double z = (v->scale > 0.0) ? v->scale : 1.0;
    *sx = (c * dx + s * dy) / z + (v->W - 1) * 0.5;
    *sy = (-s * dx + c * dy) / z + (v->H - 1) * 0.5;
}

int oracle_sizeof_view(void) { return (int)sizeof(oracle_view); }
int oracle_sizeof_kp(void) { return (int)sizeof(oracle_kp); }

/* ------------------------------------------------------------------------ */
/* Differentiable warp (the photometric refinement path) and its exact VJP   */
/* ------------------------------------------------------------------------ */
/*
 * The same chain as oracle_warp_view -- Lanczos-3 rotation (Eq. (3)-(4)),
 * Gaussian along canvas x, Lanczos-3 tilt -- with continuous parameters
 * theta = (t, phi, tx, ty) and two changes that make it C^1 in theta:
 *   - the source point is p = R(phi)^T (q - c_r) + c_s + (tx, ty) in plain
 *     floating point (the translation T of Eq. (2) acting on the source), and
 *     every tap is clamped to the image: no zero background;
 *   - the Gaussian half width K is fixed by the caller (from the largest tilt
 *     of the run), sigma = 0.8 sqrt(t^2 - 1) varies with t.
 * Canvas and view sizes are fixed (taken from the initial parameters).
 * L and L' both vanish at +-3 and the weights are normalised, so the map is
 * continuously differentiable across the switches of floor(p).
 */
typedef struct {
    int32_t W, H, Wr, Hr, Wv, Hv, K, pad;
    double t, phi, tx, ty;
} oracle_dview;

static double dsinc(double x)
{
    if (fabs(x) < 1e-4) return -(M_PI * M_PI / 3.0) * x;      /* series: -pi^2 x / 3 + O(x^3) */
    return (cos(M_PI * x) - sinc(x)) / x;
}

/* L'(x) for L(x) = sinc(x) sinc(x/3) on |x| < 3 (0 outside; L' -> 0 at +-3). */
static double lanczos3_deriv(double x)
{
    if (!(fabs(x) < 3.0)) return 0.0;
    return dsinc(x) * sinc(x / 3.0) + sinc(x) * dsinc(x / 3.0) / 3.0;
}

/* Normalised weights w_m(f) and their derivatives dw_m/df, m = -2..3. */
static void weights_and_deriv(double f, double w[6], double dw[6])
{
    double L[6], dL[6], S = 0.0, dS = 0.0;
    for (int m = -2; m <= 3; ++m) {
        L[m + 2] = oracle_lanczos3(f - m);
        dL[m + 2] = lanczos3_deriv(f - m);
        S += L[m + 2];
        dS += dL[m + 2];
    }
    for (int i = 0; i < 6; ++i) {
        w[i] = L[i] / S;
        dw[i] = (dL[i] - w[i] * dS) / S;
    }
}

/* Gaussian taps g_0..g_K at sigma (delta at sigma = 0) and dg_k/dsigma. */
static void gauss_and_deriv(double sigma, int K, double *g, double *dg)
{
    if (sigma <= 0.0) {
        for (int k = 0; k <= K; ++k) { g[k] = (k == 0); dg[k] = 0.0; }
        return;
    }
    double E = 0.0;
    for (int k = 0; k <= K; ++k) {
        g[k] = exp(-(double)k * k / (2.0 * sigma * sigma));
        E += (k == 0) ? g[k] : 2.0 * g[k];
    }
    double m2 = 0.0;
    for (int k = 0; k <= K; ++k) {
        g[k] /= E;
        m2 += (k == 0 ? 0.0 : 2.0 * g[k]) * (double)k * k;   /* sum_j g_j j^2 */
    }
    const double s3 = sigma * sigma * sigma;
    for (int k = 0; k <= K; ++k) dg[k] = g[k] * ((double)k * k - m2) / s3;
}

static void dview_src(const oracle_dview *v, int i, int j, double c, double s, double *px, double *py)
{
    const double dx = i - (v->Wr - 1) * 0.5, dy = j - (v->Hr - 1) * 0.5;
    *px = c * dx + s * dy + (v->W - 1) * 0.5 + v->tx;
    *py = -s * dx + c * dy + (v->H - 1) * 0.5 + v->ty;
}

static double dview_canvas(const double *u, const oracle_dview *v, double px, double py)
{
    const int x0 = (int)floor(px), y0 = (int)floor(py);
    double wx[6], wy[6], d6[6];
    weights_and_deriv(px - x0, wx, d6);
    weights_and_deriv(py - y0, wy, d6);
    double acc = 0.0;
    for (int n = 0; n < 6; ++n) {
        const int yy = clampi(y0 + n - 2, 0, v->H - 1);
        double row = 0.0;
        for (int m = 0; m < 6; ++m) row += wx[m] * u[(size_t)yy * v->W + clampi(x0 + m - 2, 0, v->W - 1)];
        acc += wy[n] * row;
    }
    return acc;
}

static double dview_sigma(double t) { return t > 1.0 ? 0.8 * sqrt(t * t - 1.0) : 0.0; }

/* Forward: out (Hv x Wv) = tilt(gauss(rot(u))). */
void oracle_dwarp_fwd(const double *u, const oracle_dview *v, double *out)
{
    const int Wr = v->Wr, Hr = v->Hr, Wv = v->Wv, K = v->K;
    double g[256], dg[256];
    gauss_and_deriv(dview_sigma(v->t), K, g, dg);
    const double r = v->phi * (M_PI / 180.0), c = cos(r), s = sin(r);
    double *C = (double *)malloc(sizeof(double) * (size_t)Wr);
    double *B = (double *)malloc(sizeof(double) * (size_t)Wr);
    for (int j = 0; j < Hr; ++j) {
        for (int i = 0; i < Wr; ++i) {
            double px, py;
            dview_src(v, i, j, c, s, &px, &py);
            C[i] = dview_canvas(u, v, px, py);
        }
        for (int i = 0; i < Wr; ++i) {
            double acc = 0.0;
            for (int k = -K; k <= K; ++k) acc += g[abs(k)] * C[clampi(i - k, 0, Wr - 1)];
            B[i] = acc;
        }
        for (int x = 0; x < Wv; ++x) {
            const double X = v->t * (x - (Wv - 1) * 0.5) + (Wr - 1) * 0.5;
            const int X0 = (int)floor(X);
            double w[6], d6[6];
            weights_and_deriv(X - X0, w, d6);
            double acc = 0.0;
            for (int m = 0; m < 6; ++m) acc += w[m] * B[clampi(X0 + m - 2, 0, Wr - 1)];
            out[(size_t)j * Wv + x] = acc;
        }
    }
    free(C);
    free(B);
}

/*
 * Vector-Jacobian product of oracle_dwarp_fwd: given vbar (Hv x Wv), writes
 * ubar (H x W) = J_u^T vbar and pbar = (dL/dt, dL/dphi [per degree], dL/dtx,
 * dL/dty), each step the exact transpose of its forward step (canvas and
 * blurred canvas recomputed).  dsigma/dt = 0.8 t / sqrt(t^2 - 1) enters only
 * for t > 1.
 */
void oracle_dwarp_vjp(const double *u, const oracle_dview *v, const double *vbar, double *ubar, double pbar[4])
{
    const int W = v->W, H = v->H, Wr = v->Wr, Hr = v->Hr, Wv = v->Wv, K = v->K;
    const double sigma = dview_sigma(v->t);
    double g[256], dg[256];
    gauss_and_deriv(sigma, K, g, dg);
    const double r = v->phi * (M_PI / 180.0), c = cos(r), s = sin(r);
    double *C = (double *)malloc(sizeof(double) * (size_t)Wr);
    double *B = (double *)malloc(sizeof(double) * (size_t)Wr);
    double *Bb = (double *)malloc(sizeof(double) * (size_t)Wr);
    double *Cb = (double *)malloc(sizeof(double) * (size_t)Wr);
    memset(ubar, 0, sizeof(double) * (size_t)W * H);
    double tbar = 0.0, sbar = 0.0, phibar = 0.0, txbar = 0.0, tybar = 0.0;
    for (int j = 0; j < Hr; ++j) {
        /* recompute the canvas row and its blur */
        for (int i = 0; i < Wr; ++i) {
            double px, py;
            dview_src(v, i, j, c, s, &px, &py);
            C[i] = dview_canvas(u, v, px, py);
        }
        for (int i = 0; i < Wr; ++i) {
            double acc = 0.0;
            for (int k = -K; k <= K; ++k) acc += g[abs(k)] * C[clampi(i - k, 0, Wr - 1)];
            B[i] = acc;
        }
        /* tilt: B-bar and the t-derivative through X */
        memset(Bb, 0, sizeof(double) * (size_t)Wr);
        for (int x = 0; x < Wv; ++x) {
            const double vb = vbar[(size_t)j * Wv + x];
            const double X = v->t * (x - (Wv - 1) * 0.5) + (Wr - 1) * 0.5;
            const int X0 = (int)floor(X);
            double w[6], dw[6];
            weights_and_deriv(X - X0, w, dw);
            double dvdX = 0.0;
            for (int m = 0; m < 6; ++m) {
                const int i = clampi(X0 + m - 2, 0, Wr - 1);
                Bb[i] += w[m] * vb;
                dvdX += dw[m] * B[i];
            }
            tbar += vb * dvdX * (x - (Wv - 1) * 0.5);
        }
        /* Gaussian: C-bar and the sigma-derivative */
        memset(Cb, 0, sizeof(double) * (size_t)Wr);
        for (int i = 0; i < Wr; ++i) {
            for (int k = -K; k <= K; ++k) {
                const int ic = clampi(i - k, 0, Wr - 1);
                Cb[ic] += g[abs(k)] * Bb[i];
                sbar += Bb[i] * dg[abs(k)] * C[ic];
            }
        }
        /* rotation: u-bar and the derivatives through p */
        for (int i = 0; i < Wr; ++i) {
            const double cb = Cb[i];
            if (cb == 0.0) continue;
            double px, py;
            dview_src(v, i, j, c, s, &px, &py);
            const int x0 = (int)floor(px), y0 = (int)floor(py);
            double wx[6], dwx[6], wy[6], dwy[6];
            weights_and_deriv(px - x0, wx, dwx);
            weights_and_deriv(py - y0, wy, dwy);
            double dCdx = 0.0, dCdy = 0.0;
            for (int n = 0; n < 6; ++n) {
                const int yy = clampi(y0 + n - 2, 0, H - 1);
                double row = 0.0, drow = 0.0;
                for (int m = 0; m < 6; ++m) {
                    const int xx = clampi(x0 + m - 2, 0, W - 1);
                    const double val = u[(size_t)yy * W + xx];
                    ubar[(size_t)yy * W + xx] += cb * wx[m] * wy[n];
                    row += wx[m] * val;
                    drow += dwx[m] * val;
                }
                dCdx += wy[n] * drow;
                dCdy += dwy[n] * row;
            }
            const double dx = i - (Wr - 1) * 0.5, dy = j - (Hr - 1) * 0.5;
            const double dpx_dphi = (-s * dx + c * dy) * (M_PI / 180.0);
            const double dpy_dphi = (-c * dx - s * dy) * (M_PI / 180.0);
            txbar += cb * dCdx;
            tybar += cb * dCdy;
            phibar += cb * (dCdx * dpx_dphi + dCdy * dpy_dphi);
        }
    }
    if (v->t > 1.0) tbar += sbar * 0.8 * v->t / sqrt(v->t * v->t - 1.0);
    pbar[0] = tbar;
    pbar[1] = phibar;
    pbar[2] = txbar;
    pbar[3] = tybar;
    free(C);
    free(B);
    free(Bb);
    free(Cb);
}

int oracle_sizeof_dview(void) { return (int)sizeof(oracle_dview); }

/* ------------------------------------------------------------------------ */
/* Evaluation on the accepted pairs: duplicate removal, precision (Eq. (5),  */
/* (6)), homography by RANSAC [28] and the inlier ratio (Eq. (7))            */
/* ------------------------------------------------------------------------ */
/* The accepted pairs come as four fp32 coordinate arrays (image 1 point x1,
 * y1; image 2 point x2, y2), back-projected to the original images.  Every
 * floating-point step below is a single IEEE operation in the order written
 * (compiled without contraction). */

/* Nearest integer pixel of an fp32 coordinate, floor(x + 1/2) in fp32. */
static int32_t pix_of(float x) { return (int32_t)floorf(x + 0.5f); }

/* Duplicate removal in original coordinates: pair i is kept iff no earlier
 * pair has the same four nearest pixels (x1, y1, x2, y2); keep[i] = 0/1.
 * Several views can detect the same physical correspondence, and the
 * evaluation counts each once.  Returns the number kept. */
int oracle_dedup(const float *x1, const float *y1, const float *x2, const float *y2, int n, uint8_t *keep)
{
    int kept = 0;
    for (int i = 0; i < n; ++i) {
        int dup = 0;
        for (int j = 0; j < i && !dup; ++j)
            dup = pix_of(x1[i]) == pix_of(x1[j]) && pix_of(y1[i]) == pix_of(y1[j]) &&
                  pix_of(x2[i]) == pix_of(x2[j]) && pix_of(y2[i]) == pix_of(y2[j]);
        keep[i] = (uint8_t)!dup;
        kept += !dup;
    }
    return kept;
}

/* Squared distance between H (x, y) and (u, v) (Eq. (6) before the root):
 * (x', y') = (h0 x + h1 y + h2, h3 x + h4 y + h5) / (h6 x + h7 y + h8). */
double oracle_reproj_sq(const double H[9], double x, double y, double u, double v)
{
    const double X = H[0] * x + H[1] * y + H[2];
    const double Y = H[3] * x + H[4] * y + H[5];
    const double Z = H[6] * x + H[7] * y + H[8];
    const double dx = X / Z - u, dy = Y / Z - v;
    return dx * dx + dy * dy;
}

/* Eq. (6): number of pairs whose image-1 point, mapped by the true H,
 * lands within sqrt(th_sq) of its matched image-2 point. */
int oracle_precision_count(const float *x1, const float *y1, const float *x2, const float *y2, int n,
                           const double H[9], double th_sq)
{
    int r = 0;
    for (int i = 0; i < n; ++i) r += oracle_reproj_sq(H, x1[i], y1[i], x2[i], y2[i]) <= th_sq;
    return r;
}

/* Homography from four correspondences (x_k, y_k) -> (u_k, v_k) with
 * h8 = 1: the eight linear equations
 *   h0 x + h1 y + h2 - h6 x u - h7 y u = u,  h3 x + h4 y + h5 - h6 x v - h7 y v = v
 * solved by Gaussian elimination with partial pivoting (the first row with
 * the largest |entry| in the column) and back substitution.  Returns 0 (and
 * leaves H unspecified) when a pivot is at most 1e-10 times the largest
 * |entry| of the system: collinear or coincident points. */
int oracle_homography4(const double *x, const double *y, const double *u, const double *v, double H[9])
{
    double A[8][9];
    for (int k = 0; k < 4; ++k) {
        double *r0 = A[2 * k], *r1 = A[2 * k + 1];
        r0[0] = x[k]; r0[1] = y[k]; r0[2] = 1.0; r0[3] = 0.0; r0[4] = 0.0; r0[5] = 0.0;
        r0[6] = -(x[k] * u[k]); r0[7] = -(y[k] * u[k]); r0[8] = u[k];
        r1[0] = 0.0; r1[1] = 0.0; r1[2] = 0.0; r1[3] = x[k]; r1[4] = y[k]; r1[5] = 1.0;
        r1[6] = -(x[k] * v[k]); r1[7] = -(y[k] * v[k]); r1[8] = v[k];
    }
    double amax = 0.0;
    for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 8; ++c) amax = fmax(amax, fabs(A[r][c]));
    for (int k = 0; k < 8; ++k) {
        int p = k;
        for (int r = k + 1; r < 8; ++r)
            if (fabs(A[r][k]) > fabs(A[p][k])) p = r;
        if (!(fabs(A[p][k]) > 1e-10 * amax)) return 0;
        if (p != k)
            for (int c = 0; c < 9; ++c) {
                const double tmp = A[k][c];
                A[k][c] = A[p][c];
                A[p][c] = tmp;
            }
        for (int r = k + 1; r < 8; ++r) {
            const double f = A[r][k] / A[k][k];
            for (int c = k + 1; c < 9; ++c) A[r][c] = A[r][c] - f * A[k][c];
            A[r][k] = 0.0;
        }
    }
    double h[8];
    for (int k = 7; k >= 0; --k) {
        double s = A[k][8];
        for (int c = k + 1; c < 8; ++c) s = s - A[k][c] * h[c];
        h[k] = s / A[k][k];
    }
    for (int k = 0; k < 8; ++k) {
        if (!isfinite(h[k])) return 0;
        H[k] = h[k];
    }
    H[8] = 1.0;
    return 1;
}

/* RANSAC [28] for the homography from image 1 to image 2 over n pairs.
 * Hypothesis h draws the four pairs rnd[4h + k] mod n (k = 0..3; the random
 * numbers are inputs), fits H by oracle_homography4 and counts the pairs with
 * squared reprojection error <= th_sq.  counts[h] = -1 for a hypothesis with
 * a repeated pair or a degenerate fit; Hs[9h ..] holds each fit.  The best
 * hypothesis has the largest count, the lowest h among equal counts; its
 * inliers are marked in inlier[] (Eq. (7): In_Num = their number).  Returns
 * the best h, or -1 when no hypothesis fits (n < 4 included). */
int oracle_ransac(const float *x1, const float *y1, const float *x2, const float *y2, int n, const uint32_t *rnd,
                  int n_hyp, double th_sq, int32_t *counts, double *Hs, uint8_t *inlier)
{
    int best = -1;
    for (int h = 0; h < n_hyp; ++h) {
        counts[h] = -1;
        for (int c = 0; c < 9; ++c) Hs[9 * h + c] = 0.0;
        if (n < 4) continue;
        int idx[4];
        for (int k = 0; k < 4; ++k) idx[k] = (int)(rnd[4 * h + k] % (uint32_t)n);
        int distinct = 1;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) distinct &= idx[a] != idx[b];
        if (!distinct) continue;
        double xs[4], ys[4], us[4], vs[4];
        for (int k = 0; k < 4; ++k) {
            xs[k] = x1[idx[k]];
            ys[k] = y1[idx[k]];
            us[k] = x2[idx[k]];
            vs[k] = y2[idx[k]];
        }
        if (!oracle_homography4(xs, ys, us, vs, Hs + 9 * h)) {
            for (int c = 0; c < 9; ++c) Hs[9 * h + c] = 0.0;
            continue;
        }
        counts[h] = oracle_precision_count(x1, y1, x2, y2, n, Hs + 9 * h, th_sq);
        if (best < 0 || counts[h] > counts[best]) best = h;
    }
    for (int i = 0; i < n; ++i)
        inlier[i] = (uint8_t)(best >= 0 && oracle_reproj_sq(Hs + 9 * best, x1[i], y1[i], x2[i], y2[i]) <= th_sq);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Base-image selection, Eq. (1) (Sec. III-A)                                */
/* ------------------------------------------------------------------------ */
/* Scaling coefficient from image 1 to image 2 over n matched pairs in list
 * order: f = sum over consecutive pairs i, i+1 (i + 1 < n) of
 *   (Dis(a_i, a_{i+1}) - Dis(b_i, b_{i+1})) * (1 - (Des(i) + Des(i+1)) / 1000)
 * with Dis the Euclidean pixel length of the segment in each image and Des a
 * pair's descriptor distance.  f > 0: a segment is longer in image 1, whose
 * camera is closer to the scene.  Summed in list order in fp64. */
double oracle_scale_coefficient(const float *x1, const float *y1, const float *x2, const float *y2,
                                const int32_t *des, int n)
{
    double f = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        const double da = hypot((double)x1[i + 1] - (double)x1[i], (double)y1[i + 1] - (double)y1[i]);
        const double db = hypot((double)x2[i + 1] - (double)x2[i], (double)y2[i + 1] - (double)y2[i]);
        const double w = 1.0 - (double)(des[i] + des[i + 1]) / 1000.0;
        f += (da - db) * w;
    }
    return f;
}
