"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: exact special
cases (identity, 90-degree rotations), closed forms (Gaussian attenuation of a
cosine, Harris response of a ramp, BRIEF bits of a ramp), high-precision
evaluation of Eq. (4), library routines (atan2, argmin, sorted, np.rot90) and
brute force on tiny inputs.  No GPU is needed.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2503_03479_gb300 import synth


# --------------------------------------------------------------------------
# View table: Sec. III-B sampling rule
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kmax,expected", [(2, 10), (5, 43), (6, 63)])
def test_view_count_matches_sampling_rule(kmax, expected):
    # count of j >= 0 with j*72/t < 180, t = sqrt(2)^k  <=>  4 j^2 < 25 * 2^k
    # (exact integers), one view at t = 1.
    n = 1 + sum(sum(1 for j in range(100) if 4 * j * j < 25 * 2 ** k) for k in range(1, kmax + 1))
    assert n == expected
    assert len(O.view_table(240, 320, kmax)) == expected


def test_view_geometry_matches_rotated_bbox():
    H, W = 768, 1024
    for v in O.view_table(H, W, 6):
        t = math.sqrt(2) ** v.k
        assert v.t == pytest.approx(t, rel=1e-15)
        if v.k:
            assert v.phi_deg == pytest.approx(v.j * 72 / t, rel=1e-14)
            assert v.phi_deg < 180
        # bounding box of the rotated image rectangle [-0.5, W-0.5] x [-0.5, H-0.5]
        r = math.radians(v.phi_deg)
        R = np.array([[math.cos(r), -math.sin(r)], [math.sin(r), math.cos(r)]])
        corners = np.array([[-0.5, -0.5], [W - 0.5, -0.5], [-0.5, H - 0.5], [W - 0.5, H - 0.5]]) @ R.T
        ext = corners.max(0) - corners.min(0)
        assert v.Wr == math.ceil(ext[0] - 1e-9) and v.Hr == math.ceil(ext[1] - 1e-9)
        assert v.Wv == math.ceil(v.Wr / t) and v.Hv == v.Hr
        sig = 0.8 * math.sqrt(max(t * t - 1, 0))
        assert v.sigma == pytest.approx(sig, rel=1e-14, abs=1e-15) and v.K == math.ceil(4 * sig - 1e-12)
        assert v.cq == round(math.cos(r) * 2 ** 31) or abs(v.cq - math.cos(r) * 2 ** 31) <= 0.5 + 1e-6


# --------------------------------------------------------------------------
# Lanczos kernel: Eq. (3)-(4)
# --------------------------------------------------------------------------
def test_lanczos_kernel_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(3)
    for x in np.concatenate([rng.uniform(-3.2, 3.2, 400), [1e-9, -0.5, 2.999999, 0.25]]):
        xm = mpmath.mpf(float(x))
        if abs(xm) >= 3:
            ref = 0
        else:
            ref = mpmath.sinc(mpmath.pi * xm) * mpmath.sinc(mpmath.pi * xm / 3)
        assert abs(O.lanczos3(x) - float(ref)) <= 2e-16 * max(1.0, abs(float(ref))) + 1e-16


def test_lanczos_special_values():
    assert O.lanczos3(0.0) == 1.0
    for k in (1, 2, -1, -2, 3, -3, 3.5, -7):
        assert O.lanczos3(float(k)) == 0.0


def test_lanczos_weights_sum_to_one_and_are_needed():
    raw_dev = 0.0
    for f in np.linspace(0, 1, 1001, endpoint=False):
        w = O.lanczos3_weights(f)
        assert abs(w.sum() - 1.0) <= 1e-15
        raw = sum(O.lanczos3(f - m) for m in range(-2, 4))
        raw_dev = max(raw_dev, abs(raw - 1.0))
    # raw Lanczos-3 taps do not sum to 1 (so the normalisation matters)
    assert raw_dev > 1e-3
    # symmetry at f = 1/2: w_m == w_{1-m}
    w = O.lanczos3_weights(0.5)
    assert np.allclose(w, w[::-1], atol=1e-16)
    # f = 0 is the identity
    assert np.array_equal(O.lanczos3_weights(0.0), np.array([0, 0, 1, 0, 0, 0], float))


# --------------------------------------------------------------------------
# Gaussian along the tilt axis
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_gauss_taps_sum_and_variance(k):
    t = math.sqrt(2) ** k
    sigma = 0.8 * math.sqrt(t * t - 1)
    K = math.ceil(4 * sigma)
    g = O.gauss_taps(sigma, K)
    full = np.concatenate([g[:0:-1], g])
    assert abs(full.sum() - 1) < 1e-15
    ks = np.arange(-K, K + 1)
    var = float((full * ks * ks).sum())
    # sampled Gaussian truncated at 4 sigma: variance within 0.2 % of sigma^2
    assert abs(var / sigma ** 2 - 1) < 2e-3
    assert np.all(np.diff(g) < 0)


# --------------------------------------------------------------------------
# Warp: exact special cases and a closed form
# --------------------------------------------------------------------------
def test_warp_identity_is_exact():
    u = synth.random_u8((37, 53), 11)
    v = O.view_table(37, 53, 0)[0]
    o = O.warp_view(u, v)
    assert np.array_equal(o.f64, u.astype(np.float64))
    assert np.array_equal(o.u8, u)


@pytest.mark.parametrize("phi,k", [(90.0, -1), (180.0, 2), (270.0, 1)])
def test_warp_right_angle_rotations_are_exact(phi, k):
    u = synth.random_u8((29, 41), 12)
    v = O.make_view(29, 41, 1.0, phi)
    o = O.warp_view(u, v)
    assert np.array_equal(o.f64, np.rot90(u, k).astype(np.float64))


def test_warp_constant_image_stays_constant_inside():
    u = np.full((120, 160), 77, np.uint8)
    for v in O.view_table(120, 160, 4)[1:]:
        o = O.warp_view(u, v)
        # interior: mask valid over a window wider than the Gaussian + Lanczos support
        r = int(math.ceil((v.K + 4) / v.t)) + 1
        m = o.mask.astype(bool)
        inner = m.copy()
        for s in range(1, r + 1):
            inner[:, s:] &= m[:, :-s]
            inner[:, :-s] &= m[:, s:]
        inner[:3] = inner[-3:] = False
        inner &= np.roll(m, 3, 0) & np.roll(m, -3, 0)
        assert inner.sum() > 100
        assert np.abs(o.f64[inner] - 77).max() < 1e-12


def _view_source_points(v):
    """Source coordinates of every view pixel (x', j), written independently in numpy."""
    xs = np.arange(v.Wv)
    X = v.t * (xs - (v.Wv - 1) / 2) + (v.Wr - 1) / 2
    J = np.arange(v.Hv)
    XX, JJ = np.meshgrid(X, J)
    dx, dy = XX - (v.Wr - 1) / 2, JJ - (v.Hr - 1) / 2
    r = math.radians(v.phi_deg)
    c, s = math.cos(r), math.sin(r)
    return c * dx + s * dy + (v.W - 1) / 2, -s * dx + c * dy + (v.H - 1) / 2


@pytest.mark.parametrize("t,phi", [(2.0, 30.0), (math.sqrt(2), 50.91), (2.8284271247461903, 101.8), (4.0, 162.0)])
def test_warp_cosine_closed_form(t, phi):
    """u = 128 + 100 cos(2 pi f.p): after rotation by phi the frequency in canvas
    coordinates is R(phi) f; the Gaussian along canvas x multiplies the amplitude
    by exp(-2 pi^2 sigma^2 w_x^2); the Lanczos resamplings are near-exact at this
    frequency.  Pins centres, rotation sign, tilt axis and sigma together."""
    H, W = 160, 200
    sigma = 0.8 * math.sqrt(t * t - 1)
    # frequency chosen along the canvas x axis so that the Gaussian halves it
    wx = math.sqrt(math.log(2) / (2 * math.pi ** 2 * sigma ** 2))
    wx = min(wx, 0.12)
    r = math.radians(phi)
    # p = R^T (q - c_r) + c_s, so f.p = (R f).(q - c_r) + const: the canvas
    # frequency (wx, 0) needs the source frequency f = R^T (wx, 0)
    fx, fy = math.cos(r) * wx, -math.sin(r) * wx
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    u = 128 + 100 * np.cos(2 * math.pi * (fx * xx + fy * yy) + 0.3)
    v = O.make_view(H, W, t, phi)
    o = O.warp_view(u, v)
    px, py = _view_source_points(v)
    G = math.exp(-2 * math.pi ** 2 * sigma ** 2 * wx ** 2)
    expect = 128 + 100 * G * np.cos(2 * math.pi * (fx * px + fy * py) + 0.3)
    # interior, away from the footprint edge
    m = (px > 12) & (px < W - 13) & (py > 12) & (py < H - 13)
    assert m.sum() > 500
    err = np.abs(o.f64[m] - expect[m]).max()
    assert err < 1.5, err
    # the attenuation really happened (not a sigma = 0 path)
    assert G < 0.9


def test_warp_mask_lies_inside_footprint():
    u = synth.random_u8((90, 130), 5)
    for v in O.view_table(90, 130, 3):
        o = O.warp_view(u, v)
        px, py = _view_source_points(v)
        m = o.mask.astype(bool)
        assert m.any()
        # every valid pixel's source point is inside the image (with the
        # neighbouring canvas column, at most t/2 + 1 px away)
        slack = v.t / 2 + 1e-6
        assert (px[m] >= 0.5 - slack).all() and (px[m] <= v.W - 1.5 + slack).all()
        assert (py[m] >= 0.5 - slack).all() and (py[m] <= v.H - 1.5 + slack).all()
        # every pixel well inside is valid
        deep = (px > 2 + v.t) & (px < v.W - 3 - v.t) & (py > 2 + v.t) & (py < v.H - 3 - v.t)
        assert m[deep].all()


def test_backprojection_finds_a_dot():
    H, W = 120, 140
    u = np.zeros((H, W), np.float64)
    yy, xx = np.mgrid[0:H, 0:W]
    cx, cy = 61.3, 57.8
    u = 200 * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * 3.0 ** 2))
    for v in O.view_table(H, W, 3):
        o = O.warp_view(u, v)
        j, i = np.unravel_index(np.argmax(o.f64), o.f64.shape)
        sx, sy = O.backproject(v, 0, float(i), float(j))
        # the brightest view pixel maps back within half a view pixel (t/2 px
        # along the tilt axis) of the dot
        assert math.hypot(sx - cx, sy - cy) <= v.t / 2 + 0.75


# --------------------------------------------------------------------------
# Pyramid and smoothing
# --------------------------------------------------------------------------
def test_level_sizes_round_half_up():
    for n0 in (15, 160, 186, 227, 320, 768, 1024, 3072, 4096):
        for l in range(9):
            x = Fraction(n0) * Fraction(5, 6) ** l
            assert O.level_size(n0, l) == math.floor(x + Fraction(1, 2))
    assert O.level_size(15, 1) == 13  # 12.5 rounds up


def test_downscale_constant_ramp_and_mask():
    Wp, Hp = 97, 61
    Wl, Hl = O.level_size(Wp, 1), O.level_size(Hp, 1)
    c = np.full((Hp, Wp), 131, np.uint8)
    assert (O.downscale(c, None, Wl, Hl) == 131).all()
    ramp = np.tile(np.arange(Wp, dtype=np.uint8) * 2, (Hp, 1))
    out = O.downscale(ramp, None, Wl, Hl).astype(np.float64)
    src_x = (np.arange(Wl) + 0.5) * Wp / Wl - 0.5
    inner = src_x <= Wp - 1
    # bilinear reproduces a linear function up to Q11 weights and rounding
    assert np.abs(out[:, inner] - 2 * src_x[inner]).max() <= 0.5 + 2 * 2 / 2048 + 1e-9
    m = np.ones((Hp, Wp), np.uint8)
    m[30, 40] = 0
    _, ml = O.downscale(c, m, Wl, Hl)
    bad = np.argwhere(ml == 0)
    # only output pixels whose 2x2 taps include (40, 30) are invalid
    for y, x in bad:
        sx = ((2 * x + 1) * Wp - Wl) // (2 * Wl)
        sy = ((2 * y + 1) * Hp - Hl) // (2 * Hl)
        assert sx in (39, 40) and sy in (29, 30)
    assert 1 <= len(bad) <= 4


def test_smooth_equals_library_convolution_rounded():
    ndimage = pytest.importorskip("scipy.ndimage")
    k = np.array([18, 34, 49, 54, 49, 34, 18], np.float64)
    assert k.sum() == 256
    img = synth.random_u8((45, 67), 31)
    ref = ndimage.convolve1d(img.astype(np.float64), k, axis=1, mode="nearest")
    ref = ndimage.convolve1d(ref, k, axis=0, mode="nearest")
    want = np.floor(ref / 65536.0 + 0.5).astype(np.uint8)   # exact sums, half up
    assert np.array_equal(O.smooth(img), want)


def test_smooth_preserves_constants_and_ramps_and_is_symmetric():
    c = np.full((40, 50), 200, np.uint8)
    assert (O.smooth(c) == 200).all()
    ramp = np.tile(np.arange(50, dtype=np.uint8) * 3, (40, 1))
    s = O.smooth(ramp)
    assert np.array_equal(s[:, 3:-3], ramp[:, 3:-3])
    img = synth.random_u8((33, 33), 8)
    assert np.array_equal(O.smooth(img.T.copy()), O.smooth(img).T)
    assert np.array_equal(O.smooth(img[::-1, ::-1].copy()), O.smooth(img)[::-1, ::-1])
    # the 2-D kernel has total weight 1 and a single peak (impulse response)
    imp = np.zeros((15, 15), np.uint8)
    imp[7, 7] = 255
    r = O.smooth(imp)
    assert r[7, 7] == r.max() and abs(int(r.sum()) - 255) <= 49


# --------------------------------------------------------------------------
# FAST-9
# --------------------------------------------------------------------------
def _fast_bruteforce(patch, thr):
    """Independent formulation: label the 16 circle pixels b/d/s and look for a
    run of 9 equal labels in the doubled label string."""
    circ = [(0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
            (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3)]
    c = int(patch[3, 3])
    lab = ""
    for dx, dy in circ:
        v = int(patch[3 + dy, 3 + dx])
        lab += "b" if v > c + thr else ("d" if v < c - thr else "s")
    lab2 = lab + lab
    return ("b" * 9 in lab2) or ("d" * 9 in lab2)


def test_fast_matches_bruteforce_on_random_patches():
    rng = np.random.default_rng(21)
    hits = 0
    for _ in range(4000):
        c = int(rng.integers(30, 226))
        patch = np.clip(c + rng.integers(-60, 61, size=(7, 7)) * rng.integers(0, 2, size=(7, 7)), 0, 255).astype(np.uint8)
        # bias some patches toward arcs
        if rng.uniform() < 0.5:
            s = int(rng.integers(0, 16))
            n = int(rng.integers(7, 12))
            circ = [(0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
                    (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3)]
            val = np.clip(c + int(rng.choice([-1, 1])) * int(rng.integers(15, 60)), 0, 255)
            for i in range(n):
                dx, dy = circ[(s + i) % 16]
                patch[3 + dy, 3 + dx] = val
        thr = int(rng.integers(10, 40))
        want = _fast_bruteforce(patch, thr)
        hits += want
        assert O.fast9(patch, 3, 3, thr) == want
    assert hits > 300


def test_fast_fires_on_corners_not_on_flat_edges_or_weak_noise():
    img = np.full((40, 40), 200, np.uint8)
    img[20:, 20:] = 50          # dark quadrant: convex corner at (20, 20)
    assert O.fast9(img, 20, 20, 20)
    # a pixel on a straight edge is not a corner
    assert not O.fast9(img, 30, 20, 20)
    assert not O.fast9(img, 20, 30, 20)
    # flat region and weak noise: silent
    assert not O.fast9(img, 8, 8, 20)
    rng = np.random.default_rng(2)
    noise = (128 + rng.integers(-9, 10, size=(30, 30))).astype(np.uint8)
    assert not any(O.fast9(noise, x, y, 20) for x in range(3, 27) for y in range(3, 27))
    # a small bright triangle vertex fires
    tri = np.full((40, 40), 40, np.uint8)
    for y in range(10, 30):
        tri[y, 20 - (y - 10) // 2: 21 + (y - 10) // 2] = 220
    assert O.fast9(tri, 20, 10, 20)


# --------------------------------------------------------------------------
# Harris
# --------------------------------------------------------------------------
def test_harris_closed_form_on_a_ramp():
    img = np.tile((np.arange(40) * 4).astype(np.uint8), (40, 1))
    # Ix = (1+2+1)*(4*(x+1) - 4*(x-1)) = 32, Iy = 0 on the 7x7 window
    a = 49 * 32 * 32
    assert O.harris25(img, 20, 20) == -(a * a)
    assert O.harris25(img.T.copy(), 20, 20) == -(a * a)


def test_harris_invariances_and_signs():
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, size=(21, 21), dtype=np.uint8)
    r = O.harris25(img, 10, 10)
    assert O.harris25(img.T.copy(), 10, 10) == r
    assert O.harris25(img[::-1, ::-1].copy(), 10, 10) == r
    corner = np.full((30, 30), 200, np.uint8)
    corner[15:, 15:] = 40
    assert O.harris25(corner, 15, 15) > 0
    edge = np.full((30, 30), 200, np.uint8)
    edge[:, 15:] = 40
    assert O.harris25(edge, 15, 15) < 0


# --------------------------------------------------------------------------
# Detection, NMS, quota, selection
# --------------------------------------------------------------------------
def test_detect_level_nms_properties():
    p = synth.pair_affine_small()
    img = p.img1
    H, W = img.shape
    mask = np.ones_like(img)
    xs, ys, rs = O.detect_level(img, mask)
    assert len(xs) > 50
    surv = set(zip(xs.tolist(), ys.tolist()))

    def corner(x, y):
        return 16 <= x < W - 16 and 16 <= y < H - 16 and O.fast9(img, x, y, 20)

    cache = {}
    for y in range(16, H - 16):
        for x in range(16, W - 16):
            if corner(x, y):
                cache[(x, y)] = O.harris25(img, x, y)
    for (x, y), r in cache.items():
        dominated = False
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                q = (x + dx, y + dy)
                if q == (x, y) or q not in cache:
                    continue
                rq = cache[q]
                if rq > r or (rq == r and (q[1], q[0]) < (y, x)):
                    dominated = True
        assert ((x, y) in surv) == (not dominated)
    for x, y, r in zip(xs, ys, rs):
        assert cache[(int(x), int(y))] == r


def test_nms_tie_keeps_the_raster_first_corner():
    """A mirror-symmetric image about x = 20.5 gives the corner pairs (20, y),
    (21, y) identical FAST results and equal Harris responses; of such a tied
    pair only the raster-first (left) one may survive."""
    base = synth.pair_affine_small().img1[:120, :21]
    img = np.concatenate([base, base[:, ::-1]], axis=1).copy()
    assert img.shape[1] == 42
    H, W = img.shape
    mask = np.ones_like(img)
    xs, ys, rs = O.detect_level(img, mask, thr=10)
    surv = set(zip(xs.tolist(), ys.tolist()))
    ties = 0
    for y in range(16, H - 16):
        if O.fast9(img, 20, y, 10) and O.fast9(img, 21, y, 10):
            assert O.harris25(img, 20, y) == O.harris25(img, 21, y)
            ties += 1
            assert (21, y) not in surv
    assert ties >= 1
    # the left corner of a tie survives when nothing else dominates it
    assert any((20, y) in surv for y in range(16, H - 16))


def test_quota_sums_and_proportional():
    Ws = [O.level_size(1024, l) for l in range(8)]
    Hs = [O.level_size(768, l) for l in range(8)]
    q = O.quota(Ws, Hs, 1000)
    assert q.sum() == 1000
    A = np.array(Ws) * np.array(Hs)
    assert np.all(q[1:] == (1000 * A[1:]) // A.sum())


def test_orb_selection_is_sorted_topn():
    p = synth.pair_affine_small()
    v = O.view_table(240, 320, 2)[6]
    vo = O.warp_view(p.img1, v)
    L, N = 4, 300
    o = O.orb_view(vo.u8, vo.mask, L, N)
    levels, masks = O.pyramid(vo.u8, vo.mask, L)
    q = O.quota([l.shape[1] for l in levels], [l.shape[0] for l in levels], N)
    got = o.kps
    off = 0
    for l in range(L):
        xs, ys, rs = O.detect_level(levels[l], masks[l])
        ref = sorted(zip((-rs).tolist(), ys.tolist(), xs.tolist()))[: q[l]]
        sel = got[got["level"] == l]
        assert [(-int(k["r25"]), int(k["y"]), int(k["x"])) for k in sel] == ref
        assert np.all(got["level"][off: off + len(sel)] == l)
        off += len(sel)


# --------------------------------------------------------------------------
# Orientation and descriptors
# --------------------------------------------------------------------------
def test_angle_bins_match_atan2():
    rng = np.random.default_rng(9)
    for _ in range(20000):
        mx, my = (int(v) for v in rng.integers(-2_000_000, 2_000_001, size=2))
        if mx == 0 and my == 0:
            continue
        a = math.degrees(math.atan2(my, mx)) % 360.0
        pos = (a + 6.0) / 12.0
        if abs(pos - round(pos)) < 1e-6:
            continue  # too close to a sector boundary for the double reference
        assert O.angle_bin(mx, my) == int(math.floor(pos)) % 30
    assert O.angle_bin(0, 0) == 0
    assert O.angle_bin(10, 0) == 0
    assert O.angle_bin(0, 10) == 8      # 90 deg = lower edge of sector 8
    assert O.angle_bin(-10, 0) == 15
    assert O.angle_bin(0, -10) == 23


def test_pattern_properties():
    pat = O.pattern()
    assert pat.shape == (30, 256, 4)
    base = pat[0].astype(int)
    assert ((base[:, 0] ** 2 + base[:, 1] ** 2) <= 225).all()
    assert ((base[:, 2] ** 2 + base[:, 3] ** 2) <= 225).all()
    assert not (np.all(base[:, :2] == base[:, 2:], axis=1)).any()
    assert np.array_equal(pat[15:], -pat[:15])
    # every steered copy stays inside the 31x31 patch and near the exact rotation
    for b in range(15):
        r = math.radians(12 * b)
        R = np.array([[math.cos(r), -math.sin(r)], [math.sin(r), math.cos(r)]])
        for k in (0, 2):
            ex = base[:, k:k + 2] @ R.T
            assert np.abs(pat[b][:, k:k + 2] - ex).max() <= 0.5 + 1e-9
    assert np.abs(pat).max() <= 15
    # spread of N(0, 6.2^2) truncated to the radius-15 disc
    sd = base[:, :2].std()
    assert 4.8 < sd < 6.6
    assert np.array_equal(O.pattern(), pat) and not np.array_equal(O.pattern(7), pat)


def test_brief_closed_forms():
    pat = O.pattern()
    flat = np.full((40, 40), 90, np.uint8)
    assert not O.brief(flat, 20, 20, 0, pat).any()
    ramp = np.tile(np.arange(40, dtype=np.uint8) * 5, (40, 1))
    d = O.brief(ramp, 20, 20, 0, pat)
    bits = np.unpackbits(d, bitorder="little")
    assert np.array_equal(bits, (pat[0][:, 0] < pat[0][:, 2]).astype(np.uint8))


def test_orientation_and_descriptor_under_180_rotation():
    p = synth.pair_affine_small()
    img = p.img1[:200, :280].copy()
    rot = img[::-1, ::-1].copy()
    H, W = img.shape
    sm, smr = O.smooth(img), O.smooth(rot)
    pat = O.pattern()
    rng = np.random.default_rng(1)
    for _ in range(200):
        x, y = int(rng.integers(20, W - 20)), int(rng.integers(20, H - 20))
        xr, yr = W - 1 - x, H - 1 - y
        m10, m01 = O.moments(img, x, y)
        r10, r01 = O.moments(rot, xr, yr)
        assert (r10, r01) == (-m10, -m01)
        b = O.angle_bin(m10, m01)
        br = O.angle_bin(r10, r01)
        if (m10, m01) == (0, 0):
            continue  # no orientation: both sides take bin 0
        assert br == (b + 15) % 30
        # the smoothed image commutes with the 180-degree rotation away from the borders
        assert np.array_equal(O.brief(sm, x, y, b, pat), O.brief(smr, xr, yr, br, pat))


def test_descriptor_steering_direction_under_90_rotation():
    """rot90 is exact on pixels: the moments rotate exactly and the bin moves by
    7 or 8; descriptors of corresponding points stay close only if the pattern
    is steered in the same direction as the measured angle."""
    p = synth.pair_affine_small()
    img = p.img1[:200, :200].copy()
    rot = np.rot90(img, -1).copy()       # rot[r, c] = img[H-1-c, r]
    H, W = img.shape
    sm, smr = O.smooth(img), O.smooth(rot)
    pat = O.pattern()
    rng = np.random.default_rng(5)
    dist_good, dist_bad = [], []
    for _ in range(150):
        x, y = int(rng.integers(20, W - 20)), int(rng.integers(20, H - 20))
        xr, yr = H - 1 - y, x
        m10, m01 = O.moments(img, x, y)
        r10, r01 = O.moments(rot, xr, yr)
        assert (r10, r01) == (-m01, m10)
        if abs(m10) + abs(m01) < 2000:
            continue
        b, br = O.angle_bin(m10, m01), O.angle_bin(r10, r01)
        assert (br - b) % 30 in (7, 8)
        d0 = O.brief(sm, x, y, b, pat)
        d1 = O.brief(smr, xr, yr, br, pat)
        d1_bad = O.brief(smr, xr, yr, (2 * b - br) % 30, pat)
        dist_good.append(int(np.unpackbits(d0 ^ d1).sum()))
        dist_bad.append(int(np.unpackbits(d0 ^ d1_bad).sum()))
    assert len(dist_good) > 50
    assert np.median(dist_good) < 50 and np.median(dist_bad) > 80


# --------------------------------------------------------------------------
# Matching
# --------------------------------------------------------------------------
def _bf_match(q, t, num, den):
    D = np.unpackbits(q[:, None, :] ^ t[None, :, :], axis=2).sum(2)
    best = D.argmin(1)  # first index on ties
    d1 = D[np.arange(len(q)), best]
    D2 = D.copy()
    D2[np.arange(len(q)), best] = 10 ** 6
    d2 = D2.min(1) if t.shape[0] > 1 else np.full(len(q), 257)
    acc = (t.shape[0] >= 2) & (den * d1 < num * d2)
    return best, d1, d2, acc


@pytest.mark.parametrize("nq,nt,seed", [(1, 1, 0), (7, 2, 1), (50, 64, 2), (130, 257, 3)])
def test_match_equals_bruteforce(nq, nt, seed):
    q = synth.random_descriptors(nq, seed)
    t = synth.random_descriptors(nt, seed + 100)
    # plant near-duplicates so that small distances and ties occur
    if nt > 4:
        t[3] = q[0]
        t[4] = q[0]
        t[5] = q[1] ^ np.eye(32, dtype=np.uint8)[0]
    m = O.match(q, t)
    best, d1, d2, acc = _bf_match(q, t, 4, 5)
    assert np.array_equal(m.best, best) and np.array_equal(m.d1, d1)
    assert np.array_equal(m.d2, d2) and np.array_equal(m.accepted, acc)


def test_match_self_duplicates_and_ratio_edge():
    d = synth.random_descriptors(40, 9)
    m = O.match(d, d)
    assert np.array_equal(m.best, np.arange(40)) and (m.d1 == 0).all()
    dup = np.concatenate([d, d])
    m = O.match(d, dup)
    assert not m.accepted.any() and (m.d2 == 0).all()
    # d1 = 4, d2 = 5: 5*4 < 4*5 is false -> rejected (a float32 0.8f*d2 would accept)
    q = np.zeros((1, 32), np.uint8)
    t = np.zeros((2, 32), np.uint8)
    t[0, 0] = 0b1111
    t[1, 1] = 0b11111
    m = O.match(q, t)
    assert (m.d1[0], m.d2[0], bool(m.accepted[0])) == (4, 5, False)
    t[1, 1] = 0b111111
    assert O.match(q, t).accepted[0]


# --------------------------------------------------------------------------
# End to end: reprojection with the known affine (Eq. (5)-(6))
# --------------------------------------------------------------------------
def test_end_to_end_reprojection_small_pair():
    p = synth.pair_affine_small()
    p1, p2, m = O.match_pair(p.img1, p.img2, kmax=2, L=4, N=500)
    assert len(p1.kps) > 2000 and m.accepted.sum() > 100
    x1 = p1.src_xy[m.accepted]
    x2 = p2.src_xy[m.best[m.accepted]]
    h = np.c_[x1, np.ones(len(x1))] @ p.H12.T
    err = np.hypot(*(h[:, :2] / h[:, 2:] - x2).T)
    assert np.median(err) < 1.5
    assert (err <= math.sqrt(3)).mean() >= 0.5


# --------------------------------------------------------------------------
# Scaled views (Eq. (2)'s S, the coarse stage's parameter groups)
# --------------------------------------------------------------------------
def _scaled_source_points(v):
    """Source coordinates of every view pixel of a scaled view, written
    independently in numpy: p = R^T (q - c_r) / s + c_s."""
    xs = np.arange(v.Wv)
    X = v.t * (xs - (v.Wv - 1) / 2) + (v.Wr - 1) / 2
    J = np.arange(v.Hv)
    XX, JJ = np.meshgrid(X, J)
    dx, dy = XX - (v.Wr - 1) / 2, JJ - (v.Hr - 1) / 2
    r = math.radians(v.phi_deg)
    c, s = math.cos(r), math.sin(r)
    return (c * dx + s * dy) / v.scale + (v.W - 1) / 2, (-s * dx + c * dy) / v.scale + (v.H - 1) / 2


@pytest.mark.parametrize("t,phi,scale", [(1.0, 0.0, 2.0), (2.0, 30.0, 1.5), (2.8284271247461903, 101.8, 2.0),
                                         (1.4142135623730951, 50.91, 3.5)])
def test_scaled_warp_cosine_closed_form(t, phi, scale):
    """u = 128 + 100 cos(2 pi f.p) with f = s R^T (w, 0): the canvas sees the
    frequency (w, 0) (magnified by s), the Gaussian along canvas x multiplies
    the amplitude by exp(-2 pi^2 sigma^2 w^2), the Lanczos resamplings are
    near-exact.  Pins the scale, centres and rotation of scaled views."""
    H, W = 120, 150
    sigma = 0.8 * math.sqrt(t * t - 1)
    w = 0.11 / scale                    # source frequency s w = 0.11 cycles / px
    r = math.radians(phi)
    fx, fy = scale * math.cos(r) * w, -scale * math.sin(r) * w
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    u = 128 + 100 * np.cos(2 * math.pi * (fx * xx + fy * yy) + 0.3)
    v = O.make_view(H, W, t, phi, scale)
    assert v.scale == scale
    o = O.warp_view(u, v)
    px, py = _scaled_source_points(v)
    G = math.exp(-2 * math.pi ** 2 * sigma ** 2 * w ** 2)
    expect = 128 + 100 * G * np.cos(2 * math.pi * (fx * px + fy * py) + 0.3)
    m = (px > 12) & (px < W - 13) & (py > 12) & (py < H - 13)
    assert m.sum() > 500
    err = np.abs(o.f64[m] - expect[m]).max()
    assert err < 1.5, err
    # a wrong scale (or none) misplaces the pattern by far more than that
    px1, py1 = _view_source_points(v)
    wrong = 128 + 100 * G * np.cos(2 * math.pi * (fx * px1 + fy * py1) + 0.3)
    assert np.abs(o.f64[m] - wrong[m]).max() > 20


def test_scaled_backprojection_finds_a_dot():
    H, W = 120, 140
    yy, xx = np.mgrid[0:H, 0:W]
    cx, cy = 61.3, 57.8
    u = 200 * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * 3.0 ** 2))
    for v in O.view_table_scaled(H, W, 3, 0.5):
        o = O.warp_view(u, v)
        j, i = np.unravel_index(np.argmax(o.f64), o.f64.shape)
        sx, sy = O.backproject(v, 0, float(i), float(j))
        # half a view pixel: t / (2 s) source px along the tilt axis, 1 / (2 s) across
        assert math.hypot(sx - cx, sy - cy) <= v.t / (2 * v.scale) + 0.75


def test_scaled_table_keeps_the_sampling_and_ties_s_to_k():
    a, b = O.view_table(768, 1024, 5), O.view_table_scaled(768, 1024, 5, 0.5)
    assert len(a) == len(b) == 43
    for x, y in zip(a, b):
        assert (x.k, x.j, x.t, x.phi_deg, x.sigma, x.K) == (y.k, y.j, y.t, y.phi_deg, y.sigma, y.K)
        assert x.scale == 1.0 and y.scale == 1.0 + 0.5 * y.k
        assert y.Wr >= x.Wr and y.Hr >= x.Hr
    # ds = 0 is the plain table
    for x, y in zip(a, O.view_table_scaled(768, 1024, 5, 0.0)):
        assert (x.Wr, x.Hr, x.Wv, x.cq, x.sq, x.tq) == (y.Wr, y.Hr, y.Wv, y.cq, y.sq, y.tq)


# --------------------------------------------------------------------------
# Nearest-neighbour views of the coarse stage (Sec. III-B)
# --------------------------------------------------------------------------
def test_nn_identity_and_right_angles_are_exact():
    u = synth.random_u8((29, 41), 13)
    o = O.warp_view_nn(u, O.view_table(29, 41, 0)[0])
    assert np.array_equal(o.f64, u.astype(np.float64)) and np.array_equal(o.u8, u)
    for phi, k in ((90.0, -1), (180.0, 2), (270.0, 1)):
        o = O.warp_view_nn(u, O.make_view(29, 41, 1.0, phi))
        assert np.array_equal(o.u8, np.rot90(u, k)), phi


@pytest.mark.parametrize("scale", [2, 3])
def test_nn_integer_magnification_replicates_pixels(scale):
    """phi = 0, t = 1, s integer: canvas pixel i maps to source i/s - (s-1)/(2s),
    whose nearest pixel is i // s, so the view is every pixel repeated s x s."""
    u = synth.random_u8((23, 31), 14)
    v = O.make_view(23, 31, 1.0, 0.0, float(scale))
    o = O.warp_view_nn(u, v)
    assert np.array_equal(o.u8, np.kron(u, np.ones((scale, scale), np.uint8)))


@pytest.mark.parametrize("phi,scale", [(23.0, 1.0), (61.7, 1.5), (127.3, 2.25), (200.0, 3.0)])
def test_nn_picks_a_pixel_within_half_a_pixel(phi, scale):
    """u encodes its own coordinates; at t = 1 every view pixel inside the
    footprint holds a source pixel at most half a pixel from the exact source
    point per axis (computed in floating point, not from the Q32 geometry),
    and every pixel outside holds 0."""
    H, W = 47, 59
    yy, xx = np.mgrid[0:H, 0:W]
    u = (1 + xx + 1000 * yy).astype(np.float64)
    v = O.make_view(H, W, 1.0, phi, scale)
    assert v.Wv == v.Wr and v.K == 0
    o = O.warp_view_nn(u, v)
    px, py = _scaled_source_points(v)
    eps = 1e-6
    inside = (px >= -0.5 + eps) & (px < W - 0.5 - eps) & (py >= -0.5 + eps) & (py < H - 0.5 - eps)
    outside = (px < -0.5 - eps) | (px >= W - 0.5 + eps) | (py < -0.5 - eps) | (py >= H - 0.5 + eps)
    val = o.f64.astype(np.int64)
    xs, ys = (val - 1) % 1000, (val - 1) // 1000
    assert inside.sum() > 1000
    assert (val[inside] > 0).all()
    assert (np.abs(xs[inside] - px[inside]) <= 0.5 + eps).all()
    assert (np.abs(ys[inside] - py[inside]) <= 0.5 + eps).all()
    assert (val[outside] == 0).all()


@pytest.mark.parametrize("t", [2.0, 2.8284271247461903, 4.0])
def test_nn_tilt_takes_the_nearest_blurred_column(t):
    """phi = 0, s = 1, u = 128 + 100 cos(2 pi w x): the canvas is u, the Gaussian
    along x multiplies the amplitude by exp(-2 pi^2 sigma^2 w^2), and view
    column x' takes canvas column round(t (x' - (Wv-1)/2) + (Wr-1)/2)."""
    H, W = 40, 240
    sigma = 0.8 * math.sqrt(t * t - 1)
    w = math.sqrt(math.log(2) / (2 * math.pi ** 2 * sigma ** 2))
    xx = np.broadcast_to(np.arange(W, dtype=np.float64), (H, W))
    u = 128 + 100 * np.cos(2 * math.pi * w * xx + 0.3)
    v = O.make_view(H, W, t, 0.0)
    o = O.warp_view_nn(u, v)
    X = t * (np.arange(v.Wv) - (v.Wv - 1) / 2) + (v.Wr - 1) / 2
    G = math.exp(-2 * math.pi ** 2 * sigma ** 2 * w ** 2)
    expect = 128 + 100 * G * np.cos(2 * math.pi * w * np.floor(X + 0.5) + 0.3)
    lanczos_like = 128 + 100 * G * np.cos(2 * math.pi * w * X + 0.3)
    inner = (X > 4 * sigma + 3) & (X < W - 4 * sigma - 4)
    assert inner.sum() > 20
    err = np.abs(o.f64[:, inner] - expect[inner]).max()
    assert err < 1.0, err
    # the nearest column, not the exact position
    assert np.abs(o.f64[:, inner] - lanczos_like[inner]).max() > 3.0


def test_nn_stays_near_the_lanczos_view_on_a_smooth_image():
    """On a smooth image the nearest-neighbour view differs from the (pinned)
    Lanczos-3 view by at most the gradient times the rounding distance
    (half a source pixel per axis, plus half a canvas column) where the
    Gaussian window lies inside the footprint; masks agree."""
    H, W = 110, 140
    yy, xx = np.mgrid[0:H, 0:W]
    u = 128 + 90 * np.exp(-((xx - 70.3) ** 2 + (yy - 52.6) ** 2) / (2 * 14.0 ** 2))
    gmax = 90 / (14.0 * math.sqrt(math.e))          # largest slope of the blob
    for v in O.view_table_scaled(H, W, 3, 0.5)[1:]:
        a, b = O.warp_view_nn(u, v), O.warp_view(u, v)
        assert np.array_equal(a.mask, b.mask)
        px, py = _scaled_source_points(v)
        r = (v.K + 4) * v.t / v.scale + 2
        deep = (px > r) & (px < W - 1 - r) & (py > r) & (py < H - 1 - r)
        assert deep.sum() > 50
        bound = gmax * (math.sqrt(0.5) + 0.5 / v.scale) + 0.5
        d = np.abs(a.f64[deep] - b.f64[deep])
        assert d.max() <= bound, (v.k, v.j, d.max(), bound)
        assert d.max() > 1e-3


def test_nn_constant_image_stays_constant_inside():
    u = np.full((90, 120), 181, np.uint8)
    for v in O.view_table_scaled(90, 120, 3, 0.5)[1:]:
        o = O.warp_view_nn(u, v)
        px, py = _scaled_source_points(v)
        r = (v.K + 2) * v.t / v.scale + 2
        deep = (px > r) & (px < v.W - 1 - r) & (py > r) & (py < v.H - 1 - r)
        assert deep.sum() > 50
        assert np.abs(o.f64[deep] - 181).max() < 1e-12


# --------------------------------------------------------------------------
# Evaluation on the accepted pairs: duplicates, Eq. (5)-(7), RANSAC [28]
# --------------------------------------------------------------------------
def _random_h(rng):
    return np.array([[1 + rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-20, 20)],
                     [rng.uniform(-0.2, 0.2), 1 + rng.uniform(-0.2, 0.2), rng.uniform(-20, 20)],
                     [rng.uniform(-3e-4, 3e-4), rng.uniform(-3e-4, 3e-4), 1.0]])


def _apply_h(H, pts):
    p = np.c_[pts, np.ones(len(pts))] @ H.T
    return p[:, :2] / p[:, 2:]


def test_dedup_keeps_the_first_of_each_pixel_quadruple():
    """Base pairs at distinct pixel quadruples; copies jittered inside the same
    pixels (|jitter| < 0.45) are duplicates of the earliest one."""
    rng = np.random.default_rng(70)
    base = rng.integers(0, 500, size=(60, 4)).astype(np.float64)
    base[:, 0] = np.arange(60) * 7          # distinct quadruples
    rows, want = [], []
    seen = set()
    for _ in range(400):
        b = int(rng.integers(0, 60))
        rows.append(base[b] + rng.uniform(-0.45, 0.45, 4))
        want.append(b not in seen)
        seen.add(b)
    keep = O.dedup(np.array(rows, np.float32))
    assert np.array_equal(keep, np.array(want))
    # a copy one pixel away in any coordinate is not a duplicate
    for k in range(4):
        r = np.array([base[0], base[0]], np.float32)
        r[1, k] += 1.0
        assert O.dedup(r).tolist() == [True, True]
    # the nearest pixel of a half-way coordinate is the upper one: 2.5 -> 3, -0.5 -> 0
    assert O.dedup(np.array([[2.5, 0, 0, 0], [3.4, 0, 0, 0]], np.float32)).tolist() == [True, False]
    assert O.dedup(np.array([[-0.5, 0, 0, 0], [0.49, 0, 0, 0]], np.float32)).tolist() == [True, False]


def test_precision_counts_pairs_by_planted_distance():
    """x2 = H(x1) + d (cos a, sin a) with d planted on either side of sqrt(3)."""
    rng = np.random.default_rng(71)
    H = _random_h(rng)
    p1 = rng.uniform(0, 800, size=(500, 2))
    d = np.where(rng.random(500) < 0.6, rng.uniform(0, np.sqrt(3) - 0.01, 500), rng.uniform(np.sqrt(3) + 0.01, 9, 500))
    a = rng.uniform(0, 2 * np.pi, 500)
    p2 = _apply_h(H, p1) + np.c_[d * np.cos(a), d * np.sin(a)]
    pairs = np.c_[p1, p2].astype(np.float32)
    # the fp32 storage moves the points by < 1e-4 px, far inside the 0.01 margin
    assert O.precision_count(pairs, H, 3.0) == int((d <= np.sqrt(3)).sum())
    assert O.precision_count(pairs, H, 0.0) == 0
    assert O.precision_count(pairs, H, 1e6) == 500
    # the identity on identical points: every pair, distance exactly 0
    same = np.c_[p1, p1].astype(np.float32)
    assert O.precision_count(same, np.eye(3), 0.0) == 500


def test_homography4_recovers_a_known_homography():
    rng = np.random.default_rng(72)
    for _ in range(50):
        H = _random_h(rng)
        src = rng.uniform(0, 1000, size=(4, 2))
        dst = _apply_h(H, src)
        G = O.homography4(src, dst)
        assert G is not None
        assert np.abs(G / G[2, 2] - H / H[2, 2]).max() < 1e-7
        # the order of the four correspondences does not matter
        perm = rng.permutation(4)
        G2 = O.homography4(src[perm], dst[perm])
        assert np.abs(G2 - G).max() < 1e-7 * np.abs(G).max()


def test_homography4_rejects_degenerate_samples():
    src = np.array([[0, 0], [10, 10], [20, 20], [5, 40.0]])       # three collinear
    assert O.homography4(src, src * 2) is None
    src = np.array([[0, 0], [0, 0], [20, 5], [5, 40.0]])          # coincident
    assert O.homography4(src, src + 3) is None


def _ransac_set(rng, n=300, frac=0.7, noise=0.5):
    H = _random_h(rng)
    p1 = rng.uniform(0, 900, size=(n, 2))
    inl = rng.random(n) < frac
    noise = rng.uniform(-noise, noise, size=(n, 2))
    far = rng.uniform(20, 200, n)[:, None] * np.c_[np.cos(a := rng.uniform(0, 6.3, n)), np.sin(a)]
    p2 = _apply_h(H, p1) + np.where(inl[:, None], noise, far)
    return H, np.c_[p1, p2].astype(np.float32), inl


def test_ransac_finds_the_planted_inliers():
    rng = np.random.default_rng(73)
    H, pairs, inl = _ransac_set(rng)
    rnd = rng.integers(0, 2 ** 32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    r = O.ransac(pairs, rnd, th_sq=9.0)
    assert r.best >= 0
    assert np.array_equal(r.inlier, inl)
    assert r.counts[r.best] == inl.sum() == r.counts.max()
    # Eq. (7): In_Num / Pt_Num
    assert abs(r.inlier.sum() / len(pairs) - inl.mean()) == 0
    Hb = r.Hs[r.best].reshape(3, 3)
    q = rng.uniform(100, 800, size=(20, 2))
    assert np.abs(_apply_h(Hb, q) - _apply_h(H, q)).max() < 3.0


def test_ransac_sampling_ties_and_degenerate_draws():
    rng = np.random.default_rng(74)
    H, pairs, inl = _ransac_set(rng, n=40, frac=1.0, noise=0.0)     # every fit is exact: all counts tie
    n = len(pairs)
    rnd = np.array([[1, 2, 3, 3],                 # repeated pair: no hypothesis
                    [5 + n, 9, 13 + 2 * n, 21],   # indices taken mod n
                    [9, 21, 5, 13],               # the same four pairs: the same count, later index
                    [0, 1, 2, 3],
                    [n - 1, 0, 5, 6],             # n - 1 is a pair of its own (not 0 again)
                    [2 * n, 0, 5, 6]], np.uint32) # 2n is pair 0 again
    r = O.ransac(pairs, rnd, th_sq=9.0)
    assert r.counts[0] == -1 and r.counts[5] == -1
    assert r.counts[1] == r.counts[2] == r.counts[3] == r.counts[4] == n
    assert r.best == 1                            # the lowest hypothesis among equal counts
    # fewer than four pairs: nothing to fit
    r = O.ransac(pairs[:3], rnd, th_sq=9.0)
    assert r.best == -1 and (r.counts == -1).all() and not r.inlier.any()


# --------------------------------------------------------------------------
# Lanczos-4 (8 x 8) reproduction of the best view (Sec. III-C)
# --------------------------------------------------------------------------
def test_lanczos4_kernel_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(90)
    for x in np.concatenate([rng.uniform(-4.3, 4.3, 400), [1e-9, -0.5, 3.999999, 0.25, 3.5]]):
        xm = mpmath.mpf(float(x))
        ref = 0 if abs(xm) >= 4 else mpmath.sinc(mpmath.pi * xm) * mpmath.sinc(mpmath.pi * xm / 4)
        # two library sines, two quotients and a product: a few ulp
        assert abs(O.lanczos(x, 4) - float(ref)) <= 6e-16 * max(1.0, abs(float(ref))) + 1e-16
    for k in (1, 2, 3, -3, 4, -4, 5):
        assert O.lanczos(float(k), 4) == 0.0
    assert O.lanczos(0.0, 4) == 1.0


def test_lanczos4_weights():
    raw_dev = 0.0
    for f in np.linspace(0, 1, 501, endpoint=False):
        w = O.lanczos_weights(f, 4)
        assert len(w) == 8 and abs(w.sum() - 1.0) <= 1e-15
        raw_dev = max(raw_dev, abs(sum(O.lanczos(f - m, 4) for m in range(-3, 5)) - 1.0))
    assert raw_dev > 1e-4
    assert np.allclose(O.lanczos_weights(0.5, 4), O.lanczos_weights(0.5, 4)[::-1], atol=1e-16)
    assert np.array_equal(O.lanczos_weights(0.0, 4), np.eye(8)[3])
    # a = 3 is the 6-tap rule of the main path
    for f in (0.0, 0.13, 0.5, 0.91):
        assert np.array_equal(O.lanczos_weights(f, 3), O.lanczos3_weights(f))


def test_lanczos4_view_exact_cases():
    u = synth.random_u8((31, 45), 91)
    o = O.warp_view_lanczos(u, O.view_table(31, 45, 0)[0], 4)
    assert np.array_equal(o.f64, u.astype(np.float64))
    for phi, k in ((90.0, -1), (180.0, 2), (270.0, 1)):
        o = O.warp_view_lanczos(u, O.make_view(31, 45, 1.0, phi), 4)
        assert np.array_equal(o.f64, np.rot90(u, k).astype(np.float64))


@pytest.mark.parametrize("t,phi,scale", [(2.0, 30.0, 1.0), (2.8284271247461903, 101.8, 1.0), (4.0, 162.0, 1.5)])
def test_lanczos4_view_cosine_closed_form(t, phi, scale):
    """As the Lanczos-3 closed form: the blurred cosine at the exact source
    points; Lanczos-4 resamples a cosine of 0.11 cycles/px more closely than
    Lanczos-3 does."""
    H, W = 140, 180
    sigma = 0.8 * math.sqrt(t * t - 1)
    w = 0.11 / scale
    r = math.radians(phi)
    fx, fy = scale * math.cos(r) * w, -scale * math.sin(r) * w
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    u = 128 + 100 * np.cos(2 * math.pi * (fx * xx + fy * yy) + 0.3)
    v = O.make_view(H, W, t, phi, scale)
    px, py = _scaled_source_points(v)
    G = math.exp(-2 * math.pi ** 2 * sigma ** 2 * w ** 2)
    expect = 128 + 100 * G * np.cos(2 * math.pi * (fx * px + fy * py) + 0.3)
    m = (px > 14) & (px < W - 15) & (py > 14) & (py < H - 15)
    assert m.sum() > 500
    e4 = np.abs(O.warp_view_lanczos(u, v, 4).f64[m] - expect[m]).max()
    e3 = np.abs(O.warp_view(u, v).f64[m] - expect[m]).max()
    assert e4 < 1.5, e4
    assert e4 < e3


def test_lanczos_a3_is_the_main_view_and_a4_differs():
    u = synth.texture(90, 120, 92)
    for v in O.view_table_scaled(90, 120, 2, 0.5)[1:]:
        a3 = O.warp_view_lanczos(u, v, 3)
        ref = O.warp_view(u, v)
        assert np.array_equal(a3.f64, ref.f64) and np.array_equal(a3.mask, ref.mask)
        a4 = O.warp_view_lanczos(u, v, 4)
        assert np.array_equal(a4.mask, ref.mask)
        assert np.abs(a4.f64 - ref.f64).max() > 0.1


# --------------------------------------------------------------------------
# Base-image selection: Eq. (1)
# --------------------------------------------------------------------------
def _pairs_from(p1, p2, des):
    pairs = np.zeros(len(p1), np.dtype([("x1", np.float32), ("y1", np.float32), ("x2", np.float32),
                                         ("y2", np.float32), ("d1", np.uint16)]))
    pairs["x1"], pairs["y1"] = p1[:, 0], p1[:, 1]
    pairs["x2"], pairs["y2"] = p2[:, 0], p2[:, 1]
    pairs["d1"] = des
    return pairs


def test_scale_coefficient_closed_form_under_a_similarity():
    """Image 2 = image 1 scaled by k (rotated and shifted): every segment is k
    times as long in image 2, so f = (1 - k) sum_i Dis(a_i, a_i+1) w_i, with
    the weights w_i = 1 - (Des(i) + Des(i+1)) / 1000."""
    rng = np.random.default_rng(95)
    p1 = rng.uniform(0, 500, size=(300, 2)).astype(np.float32).astype(np.float64)
    des = rng.integers(0, 120, 300)
    for k in (0.5, 0.8, 1.0, 1.25, 2.0):
        th = 0.7
        R = k * np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        p2 = p1 @ R.T + np.array([13.0, -7.0])
        pairs = _pairs_from(p1, p2, des)
        seg = np.hypot(*np.diff(p1, axis=0).T)
        w = 1 - (des[:-1] + des[1:]) / 1000.0
        expect = (1 - k) * float((seg * w).sum())
        f = O.scale_coefficient(pairs)
        # the fp32 storage of image 2's points moves each length by < 1e-4
        assert abs(f - expect) <= 1e-4 * len(p1) + 1e-9 * abs(expect), (k, f, expect)
        if k < 1:
            assert f > 0          # image 1 shows the scene larger: it is the closer camera
        if k > 1:
            assert f < 0


def test_scale_coefficient_weights_and_degenerate_lists():
    p1 = np.array([[0, 0], [3, 4], [3, 10]], np.float64)
    p2 = np.array([[0, 0], [0, 0], [0, 0]], np.float64)
    # segments of length 5 and 6, weights 1 - (10 + 20)/1000 and 1 - (20 + 40)/1000
    f = O.scale_coefficient(_pairs_from(p1, p2, np.array([10, 20, 40])))
    assert abs(f - (5 * 0.97 + 6 * 0.94)) < 1e-12
    assert O.scale_coefficient(_pairs_from(p1[:1], p2[:1], np.array([3]))) == 0.0
    assert O.scale_coefficient(_pairs_from(p1[:0], p2[:0], np.zeros(0, int))) == 0.0
