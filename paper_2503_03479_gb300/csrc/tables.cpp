// tables.cpp -- host-side tables of libasift, generated from their written
// definitions (compiled without FMA contraction so that every double result
// is the plain IEEE evaluation of the stated expression).
//
//  * view descriptors: sampling rule of Sec. III-B (t = sqrt2^k, phi = j 72/t
//    degrees < 180, one view at t = 1), Eq. (2) geometry with psi = 0, s = 1;
//    Gaussian sigma = 0.8 sqrt(t^2 - 1) truncated at K = ceil(4 sigma);
//  * pyramid sizes: round-half-up(n0 (5/6)^l) in exact integers;
//  * steered rBRIEF-256 pattern: SplitMix64 -> Box-Muller N(0, (31/5)^2),
//    ties-to-even rounding, radius-15 disc, p != q; rotations by b * 12 deg
//    rounded half away from zero for b < 15, negated copies for b >= 15;
//  * orientation sectors: Q30 unit vectors at b * 12 - 6 deg, negated for b >= 15.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "kernels.h"

namespace asift {

namespace {

constexpr double kPi = 3.14159265358979323846;

// sin / cos of an angle in degrees; exact at multiples of 90 degrees.
void deg_sincos(double deg, double &s, double &c)
{
    const double q = deg / 90.0;
    if (std::fmod(deg, 90.0) == 0.0) {
        const long k = (((long)q % 4) + 4) % 4;
        s = (k == 1) ? 1.0 : (k == 3 ? -1.0 : 0.0);
        c = (k == 0) ? 1.0 : (k == 2 ? -1.0 : 0.0);
        return;
    }
    const double r = deg * (kPi / 180.0);
    s = std::sin(r);
    c = std::cos(r);
}

double tilt(int k)
{
    const double base = (k % 2 == 0) ? 1.0 : std::sqrt(2.0);
    return std::ldexp(base, k / 2);
}

uint64_t splitmix_next(uint64_t &state)
{
    state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double unit_open0(uint64_t &state)   // uniform in (0, 1]
{
    return (double)((splitmix_next(state) >> 11) + 1) * 0x1.0p-53;
}

}  // namespace

void make_view_desc(int H, int W, double t, double phi_deg, int k, int j, double scale, asift_view_desc *v)
{
    std::memset(v, 0, sizeof(*v));
    double s, c;
    deg_sincos(phi_deg, s, c);
    v->k = k;
    v->j = j;
    v->W = W;
    v->H = H;
    v->t = t;
    v->phi_deg = phi_deg;
    v->s = scale;
    // the canvas is the bounding box of the rotated image magnified by scale
    v->Wr = (int32_t)std::ceil(scale * ((double)W * std::fabs(c) + (double)H * std::fabs(s)) - 1e-9);
    v->Hr = (int32_t)std::ceil(scale * ((double)W * std::fabs(s) + (double)H * std::fabs(c)) - 1e-9);
    v->Wv = (int32_t)std::ceil((double)v->Wr / t);
    v->Hv = v->Hr;
    v->sigma = (t == 1.0) ? 0.0 : 0.8 * std::sqrt(t * t - 1.0);
    v->K = (int32_t)std::ceil(4.0 * v->sigma);
    v->cq = std::llrint(c / scale * 2147483648.0);
    v->sq = std::llrint(s / scale * 2147483648.0);
    v->tq = std::llrint(t * 2147483648.0);
    if (v->K == 0) {
        v->g[0] = 1.0f;
    } else {
        double g[ASIFT_MAX_GAUSS];
        double total = 0.0;
        for (int i = 0; i <= v->K && i < ASIFT_MAX_GAUSS; ++i) {
            g[i] = std::exp(-(double)i * (double)i / (2.0 * v->sigma * v->sigma));
            total += (i == 0) ? g[i] : 2.0 * g[i];
        }
        for (int i = 0; i <= v->K && i < ASIFT_MAX_GAUSS; ++i) v->g[i] = (float)(g[i] / total);
    }
}

int view_table_scaled(int H, int W, int kmax, double ds, asift_view_desc *out, int cap)
{
    int n = 0;
    for (int k = 0; k <= kmax; ++k) {
        const double t = tilt(k);
        const int jmax = (k == 0) ? 1 : 1 << 20;
        for (int j = 0; j < jmax; ++j) {
            const double phi = (k == 0) ? 0.0 : (double)j * 72.0 / t;
            if (!(phi < 180.0)) break;
            if (out && n < cap) make_view_desc(H, W, t, phi, k, j, 1.0 + (double)k * ds, &out[n]);
            ++n;
        }
    }
    return n;
}

int view_table(int H, int W, int kmax, asift_view_desc *out, int cap) { return view_table_scaled(H, W, kmax, 0.0, out, cap); }

int level_size(int n0, int l)
{
    long long num = 2LL * n0, den = 2;
    for (int i = 0; i < l; ++i) { num *= 5; den *= 6; }
    return (int)((num + den / 2) / den);
}

void make_pattern(uint64_t seed, int8_t pat[30][256][4])
{
    uint64_t st = seed;
    int pts[256][4];
    const double sd = 31.0 / 5.0;
    int have = 0;
    while (have < 256) {
        int xy[2][2];
        int got = 0;
        while (got < 2) {
            const double u1 = unit_open0(st);
            const double u2 = unit_open0(st);
            const double rad = std::sqrt(-2.0 * std::log(u1));
            const double ang = 2.0 * kPi * u2;
            const int x = (int)std::nearbyint(sd * rad * std::cos(ang));
            const int y = (int)std::nearbyint(sd * rad * std::sin(ang));
            if (x * x + y * y > 225) continue;
            xy[got][0] = x;
            xy[got][1] = y;
            ++got;
        }
        if (xy[0][0] == xy[1][0] && xy[0][1] == xy[1][1]) continue;
        pts[have][0] = xy[0][0];
        pts[have][1] = xy[0][1];
        pts[have][2] = xy[1][0];
        pts[have][3] = xy[1][1];
        ++have;
    }
    for (int b = 0; b < 15; ++b) {
        double s, c;
        deg_sincos((double)b * 12.0, s, c);
        for (int i = 0; i < 256; ++i) {
            for (int h = 0; h < 4; h += 2) {
                const double x = pts[i][h], y = pts[i][h + 1];
                const int rx = (int)std::round(c * x - s * y);
                const int ry = (int)std::round(s * x + c * y);
                pat[b][i][h] = (int8_t)rx;
                pat[b][i][h + 1] = (int8_t)ry;
                pat[b + 15][i][h] = (int8_t)-rx;
                pat[b + 15][i][h + 1] = (int8_t)-ry;
            }
        }
    }
}

void make_bin_table(long long e[30][2])
{
    for (int b = 0; b < 15; ++b) {
        double s, c;
        deg_sincos((double)b * 12.0 - 6.0, s, c);
        e[b][0] = std::llrint(c * 1073741824.0);
        e[b][1] = std::llrint(s * 1073741824.0);
        e[b + 15][0] = -e[b][0];
        e[b + 15][1] = -e[b][1];
    }
}

}  // namespace asift
