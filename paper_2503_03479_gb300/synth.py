"""Seeded synthetic image generators shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the feature-matching method itself: it only
renders textured test images and known geometric transforms between them.  The
paper measures on the Mikolajczyk and MorelYu image sets (Sec. IV-A); these
generators stand in for them with images of the same kind (8-bit grayscale,
planar textured scenes seen under large tilts).

Recipe (one definition, used everywhere):
  * texture: white Gaussian noise -> FFT -> amplitude * 1/max(|f|, 1/64 cyc/px)
    -> inverse FFT -> mean 128, std 40; then 20 + area/20000 opaque filled
    ellipses and convex polygons (3-8 vertices) with uniform grey levels;
    clip and round to uint8.
  * second image of a pair: the first image (or a larger canonical texture)
    resampled through a known homography with 4x4 supersampled bilinear
    interpolation in fp64, background 128, optional N(0, sigma^2) noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# The shapes are drawn row by row: along a row a convex shape covers an
# interval, found in closed form.  Columns more than a safe margin inside it
# are filled directly; only the few columns near its two ends are decided by
# the shape's own membership test (the same floating-point expression for
# every pixel), so the result is the membership test applied to every pixel
# of the bounding box, at a cost that grows with the shape's perimeter
# rather than its area.

def _paint_rows(img, y0, x0, x1, sa, sb, ca, cb, exact, grey):
    """Rows y0 .. y0 + len(sa) - 1 of img: columns [sa, sb] are inside, the
    columns of [ca, cb] outside [sa, sb] are decided by exact(yy, xx) (float
    arrays of pixel coordinates), all other columns of [x0, x1) are outside."""
    n = len(sa)
    if n == 0:
        return
    sa = np.clip(sa, x0, x1).astype(np.int64)
    sb = np.clip(sb, x0 - 1, x1 - 1).astype(np.int64)
    ca = np.clip(ca, x0, x1).astype(np.int64)
    cb = np.clip(cb, x0 - 1, x1 - 1).astype(np.int64)
    empty = sb < sa
    sa = np.where(empty, cb + 1, sa)     # no sure interior: the whole candidate range is tested
    sb = np.where(empty, cb, sb)
    cols = np.arange(x0, x1, dtype=np.int64)[None, :]
    sure = (cols >= sa[:, None]) & (cols <= sb[:, None])
    # boundary columns: [ca, sa - 1] and [sb + 1, cb]
    left = np.maximum(sa - ca, 0)
    right = np.maximum(cb - sb, 0)
    rows = np.arange(n)
    ry = np.concatenate([np.repeat(rows, left), np.repeat(rows, right)])
    off_l = np.arange(int(left.sum())) - np.repeat(np.cumsum(left) - left, left)
    off_r = np.arange(int(right.sum())) - np.repeat(np.cumsum(right) - right, right)
    rx = np.concatenate([np.repeat(ca, left) + off_l, np.repeat(sb + 1, right) + off_r])
    if len(ry):
        inside = exact((ry + y0).astype(np.float64), rx.astype(np.float64))
        sure[ry[inside], rx[inside] - x0] = True
    img[y0:y0 + n, x0:x1][sure] = grey


def _fill_ellipse(img, rng):
    H, W = img.shape
    cx, cy = rng.uniform(0, W), rng.uniform(0, H)
    a = rng.uniform(4, max(6.0, min(W, H) / 6))
    b = rng.uniform(4, max(6.0, min(W, H) / 6))
    th = rng.uniform(0, math.pi)
    grey = rng.uniform(0, 255)
    r = int(math.ceil(max(a, b))) + 1
    x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
    y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
    if x0 >= x1 or y0 >= y1:
        return
    c, s = math.cos(th), math.sin(th)

    def exact(yy, xx):
        dx, dy = xx - cx, yy - cy
        u = (dx * c + dy * s) / a
        v = (-dx * s + dy * c) / b
        return u * u + v * v <= 1.0

    # along row y the test is A dx^2 + B dx + C <= 0 (dx = x - cx): its roots
    # are dxm -+ w; one pixel beyond them the quadratic is at least A > 0
    # away from 0, far above the rounding of the test
    dy = np.arange(y0, y1, dtype=np.float64) - cy
    qa = c * c / (a * a) + s * s / (b * b)
    qb = 2.0 * dy * c * s * (1.0 / (a * a) - 1.0 / (b * b))
    qc = dy * dy * (s * s / (a * a) + c * c / (b * b)) - 1.0
    disc = qb * qb - 4.0 * qa * qc
    dxm = -qb / (2.0 * qa)
    w = np.sqrt(np.maximum(disc, 0.0)) / (2.0 * qa)
    sa = np.ceil(cx + dxm - w + 1.0)
    sb = np.floor(cx + dxm + w - 1.0)
    ca = np.floor(cx + dxm - w - 1.0)
    cb = np.ceil(cx + dxm + w + 1.0)
    _paint_rows(img, y0, x0, x1, sa, sb, ca, cb, exact, grey)


def _fill_polygon(img, rng):
    H, W = img.shape
    n = int(rng.integers(3, 9))
    cx, cy = rng.uniform(0, W), rng.uniform(0, H)
    rad = rng.uniform(5, max(8.0, min(W, H) / 5))
    ang = np.sort(rng.uniform(0, 2 * math.pi, n))
    px = cx + rad * np.cos(ang)
    py = cy + rad * np.sin(ang)
    grey = rng.uniform(0, 255)
    x0, x1 = max(0, int(px.min())), min(W, int(px.max()) + 2)
    y0, y1 = max(0, int(py.min())), min(H, int(py.max()) + 2)
    if x0 >= x1 or y0 >= y1:
        return
    # vertices sorted by angle around an interior point -> counter-clockwise
    # convex polygon; a point is inside iff it is left of every edge.
    edges = [(px[k], py[k], px[(k + 1) % n], py[(k + 1) % n]) for k in range(n)]

    def exact(yy, xx):
        inside = np.ones(xx.shape, dtype=bool)
        for ax, ay, bx, by in edges:
            inside &= (bx - ax) * (yy - ay) - (by - ay) * (xx - ax) >= 0
        return inside

    # edge k along row y: cross(x) = e - beta (x - ax), beta = by - ay.  The
    # sure interior keeps cross >= tau for every edge, the candidates cross >=
    # -tau; tau = 1e-6 is far above the rounding of the test (its terms stay
    # below 1e8 in magnitude)
    tau = 1e-6
    yy = np.arange(y0, y1, dtype=np.float64)
    lo_s = np.full(len(yy), -np.inf)
    hi_s = np.full(len(yy), np.inf)
    lo_c, hi_c = lo_s.copy(), hi_s.copy()
    for ax, ay, bx, by in edges:
        e = (bx - ax) * (yy - ay)
        beta = by - ay
        if beta > 0:
            hi_s = np.minimum(hi_s, ax + (e - tau) / beta)
            hi_c = np.minimum(hi_c, ax + (e + tau) / beta)
        elif beta < 0:
            lo_s = np.maximum(lo_s, ax + (e - tau) / beta)
            lo_c = np.maximum(lo_c, ax + (e + tau) / beta)
        else:
            hi_s = np.where(e >= tau, hi_s, -np.inf)
            hi_c = np.where(e >= -tau, hi_c, -np.inf)
    big = float(W + 4)
    sa = np.ceil(np.clip(lo_s, -big, big))
    sb = np.floor(np.clip(hi_s, -big, big))
    ca = np.floor(np.clip(lo_c, -big, big))
    cb = np.ceil(np.clip(hi_c, -big, big))
    _paint_rows(img, y0, x0, x1, sa, sb, ca, cb, exact, grey)


def texture(H: int, W: int, seed: int) -> np.ndarray:
    """Seeded 1/f-noise texture with opaque shapes, uint8 (H, W)."""
    rng = _rng(seed)
    noise = rng.standard_normal((H, W))
    F = np.fft.fft2(noise)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    F *= 1.0 / np.maximum(f, 1.0 / 64.0)
    img = np.real(np.fft.ifft2(F))
    img = (img - img.mean()) / (img.std() + 1e-12) * 40.0 + 128.0
    n_shapes = 20 + (H * W) // 20000
    for _ in range(n_shapes):
        if rng.uniform() < 0.5:
            _fill_ellipse(img, rng)
        else:
            _fill_polygon(img, rng)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def render(src: np.ndarray, Hmat: np.ndarray, out_shape, ss: int = 4,
           bg: float = 128.0, chunk_rows: int = 64) -> np.ndarray:
    """Resample ``src`` (uint8 or float) so that out(q) = src(Hmat^-1 q).

    ``Hmat`` is a 3x3 homography from source pixel coordinates to output pixel
    coordinates (pixel centres at integers).  Each output pixel averages ss*ss
    bilinear samples in fp64; samples outside the source take ``bg``.
    Returns float64.
    """
    Hh, Ww = out_shape
    Hinv = np.linalg.inv(Hmat)
    s = src.astype(np.float64)
    sh, sw = s.shape
    offs = (np.arange(ss) + 0.5) / ss - 0.5
    out = np.empty((Hh, Ww), dtype=np.float64)
    for r0 in range(0, Hh, chunk_rows):
        r1 = min(Hh, r0 + chunk_rows)
        yy, xx = np.mgrid[r0:r1, 0:Ww].astype(np.float64)
        acc = np.zeros(yy.shape)
        for oy in offs:
            for ox in offs:
                qx, qy = xx + ox, yy + oy
                den = Hinv[2, 0] * qx + Hinv[2, 1] * qy + Hinv[2, 2]
                px = (Hinv[0, 0] * qx + Hinv[0, 1] * qy + Hinv[0, 2]) / den
                py = (Hinv[1, 0] * qx + Hinv[1, 1] * qy + Hinv[1, 2]) / den
                inside = (px >= 0) & (px <= sw - 1) & (py >= 0) & (py <= sh - 1)
                x0 = np.clip(np.floor(px), 0, sw - 2).astype(np.int64)
                y0 = np.clip(np.floor(py), 0, sh - 2).astype(np.int64)
                fx = np.clip(px - x0, 0, 1)
                fy = np.clip(py - y0, 0, 1)
                v = ((1 - fx) * (1 - fy) * s[y0, x0] + fx * (1 - fy) * s[y0, x0 + 1]
                     + (1 - fx) * fy * s[y0 + 1, x0] + fx * fy * s[y0 + 1, x0 + 1])
                acc += np.where(inside, v, bg)
        out[r0:r1] = acc / (ss * ss)
    return out


def _rot(deg: float) -> np.ndarray:
    r = math.radians(deg)
    c, s = math.cos(r), math.sin(r)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _trans(tx: float, ty: float) -> np.ndarray:
    return np.array([[1.0, 0.0, tx], [0.0, 1.0, ty], [0.0, 0.0, 1.0]])


def _scale(sx: float, sy: float) -> np.ndarray:
    return np.diag([sx, sy, 1.0])


def tilt_about_centre(shape_in, shape_out, t: float, phi_deg: float,
                      zoom: float = 1.0) -> np.ndarray:
    """Homography (affine) that rotates by phi, compresses x by t and zooms,
    mapping the centre of an input of ``shape_in`` to the centre of ``shape_out``."""
    hi, wi = shape_in
    ho, wo = shape_out
    return (_trans((wo - 1) / 2, (ho - 1) / 2) @ _scale(zoom / t, zoom)
            @ _rot(phi_deg) @ _trans(-(wi - 1) / 2, -(hi - 1) / 2))


def perspective_tilt(shape_in, shape_out, t: float, phi_deg: float,
                     zoom: float = 1.0, persp: float = 0.0) -> np.ndarray:
    """A homography whose local affine part at the output centre is a tilt t
    along direction phi (plus a mild perspective term along that direction)."""
    A = tilt_about_centre(shape_in, shape_out, t, phi_deg, zoom)
    ho, wo = shape_out
    # perspective row acting along the (rotated) x axis of the output
    P = (_trans((wo - 1) / 2, (ho - 1) / 2)
         @ np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [persp, 0.0, 1.0]])
         @ _trans(-(wo - 1) / 2, -(ho - 1) / 2))
    return P @ A


@dataclass
class Pair:
    img1: np.ndarray          # uint8 (H1, W1)
    img2: np.ndarray          # uint8 (H2, W2)
    H12: np.ndarray           # 3x3: img1 pixel coords -> img2 pixel coords
    name: str


def pair_affine_small(seed: int = 1000, H: int = 240, W: int = 320,
                      t: float = 2.0, phi_deg: float = 30.0) -> Pair:
    """320x240 texture; image 2 = image 1 under tilt 2 after a 30 deg rotation."""
    img1 = texture(H, W, seed)
    A = tilt_about_centre((H, W), (H, W), t, phi_deg)
    img2 = np.clip(np.rint(render(img1, A, (H, W))), 0, 255).astype(np.uint8)
    return Pair(img1, img2, A, f"affine_{W}x{H}_t{t}_phi{phi_deg}")


def pair_extreme_tilt(seed: int = 2000, H: int = 768, W: int = 1024,
                      t1: float = 2.97, t2: float = 1 / math.cos(math.radians(75)),
                      phi1: float | None = None, noise_sigma: float = 2.0, ss: int = 4) -> Pair:
    """A large canonical texture seen twice: image 1 with absolute tilt t1 along
    phi1, image 2 under a homography with local tilt t2 along phi1 + 90 deg
    (transition tilt t1*t2), plus Gaussian noise on image 2.  ss: supersampling
    per axis of the rendering."""
    rng = _rng(seed + 7)
    if phi1 is None:
        phi1 = float(rng.uniform(0, 180))
    tex = texture(2 * H, 2 * W, seed)
    # magnify so that the tilted footprint stays inside the 2x texture
    zoom1 = max(1.0, max(t1, t2) / 2.0)
    zoom2 = zoom1
    A1 = tilt_about_centre(tex.shape, (H, W), t1, phi1, zoom1)
    H2 = perspective_tilt(tex.shape, (H, W), t2, phi1 + 90.0, zoom2, persp=1e-4)
    img1 = np.clip(np.rint(render(tex, A1, (H, W), ss=ss)), 0, 255).astype(np.uint8)
    im2 = render(tex, H2, (H, W), ss=ss)
    if noise_sigma > 0:
        im2 = im2 + rng.standard_normal(im2.shape) * noise_sigma
    img2 = np.clip(np.rint(im2), 0, 255).astype(np.uint8)
    return Pair(img1, img2, H2 @ np.linalg.inv(A1), f"tilt_{W}x{H}_t{t1:.2f}x{t2:.2f}")


def pairs_mixed(seed: int, n_pairs: int, wmin=480, wmax=1920, hmin=360, hmax=1080,
                tilt_deg=(30.0, 85.0)) -> list[Pair]:
    """Pairs of uneven sizes with absolute tilts drawn from ``tilt_deg``."""
    rng = _rng(seed)
    out = []
    for p in range(n_pairs):
        W = int(rng.integers(wmin, wmax + 1))
        H = int(rng.integers(hmin, hmax + 1))
        a1, a2 = rng.uniform(*tilt_deg, size=2)
        t1 = 1 / math.cos(math.radians(a1))
        t2 = 1 / math.cos(math.radians(a2))
        tex = texture(2 * H, 2 * W, seed * 1000 + p)
        phi1, phi2 = rng.uniform(0, 180, size=2)
        zoom = max(1.0, max(t1, t2) / 2.0)
        A1 = tilt_about_centre(tex.shape, (H, W), t1, phi1, zoom)
        A2 = tilt_about_centre(tex.shape, (H, W), t2, phi2, zoom)
        img1 = np.clip(np.rint(render(tex, A1, (H, W), ss=2)), 0, 255).astype(np.uint8)
        img2 = np.clip(np.rint(render(tex, A2, (H, W), ss=2)), 0, 255).astype(np.uint8)
        out.append(Pair(img1, img2, A2 @ np.linalg.inv(A1), f"mixed_{p}_{W}x{H}"))
    return out


def mixed_pair(seed: int, index: int, wmin=480, wmax=1920, hmin=360, hmax=1080,
               tilt_deg=(30.0, 85.0), ss: int = 2) -> Pair:
    """Pair `index` of a mixed-size batch, generated independently of the
    others (so a batch can be built in parallel): size uniform in
    [wmin, wmax] x [hmin, hmax], absolute tilts of both images uniform in
    ``tilt_deg``, random longitudes, a 2x canonical texture."""
    rng = _rng(seed * 100003 + index)
    W = int(rng.integers(wmin, wmax + 1))
    H = int(rng.integers(hmin, hmax + 1))
    a1, a2 = rng.uniform(*tilt_deg, size=2)
    t1 = 1 / math.cos(math.radians(a1))
    t2 = 1 / math.cos(math.radians(a2))
    phi1, phi2 = rng.uniform(0, 180, size=2)
    tex = texture(2 * H, 2 * W, seed * 1000 + index)
    zoom = max(1.0, max(t1, t2) / 2.0)
    A1 = tilt_about_centre(tex.shape, (H, W), t1, phi1, zoom)
    A2 = tilt_about_centre(tex.shape, (H, W), t2, phi2, zoom)
    img1 = np.clip(np.rint(render(tex, A1, (H, W), ss=ss)), 0, 255).astype(np.uint8)
    img2 = np.clip(np.rint(render(tex, A2, (H, W), ss=ss)), 0, 255).astype(np.uint8)
    return Pair(img1, img2, A2 @ np.linalg.inv(A1), f"mixed_{index}_{W}x{H}")


def random_u8(shape, seed: int) -> np.ndarray:
    return _rng(seed).integers(0, 256, size=shape, dtype=np.uint8)


def random_descriptors(n: int, seed: int) -> np.ndarray:
    """n x 32 uint8 random 256-bit descriptors."""
    return _rng(seed).integers(0, 256, size=(n, 32), dtype=np.uint8)


def large_pair(seed: int, index: int, H: int = 3072, W: int = 4096, ss: int = 1) -> Pair:
    """Pair `index` of the large extreme-tilt batch: pair_extreme_tilt at
    H x W with absolute tilts t1, t2 drawn from [1/cos 60 deg, 1/cos 83 deg]
    (t up to 8.2), generated independently of the other pairs."""
    rng = _rng(seed * 1000 + index)
    tmax = 1 / math.cos(math.radians(83))
    t1 = float(rng.uniform(2.0, tmax))
    t2 = float(rng.uniform(2.0, tmax))
    return pair_extreme_tilt(seed * 1000 + index, H, W, t1=t1, t2=t2, ss=ss)

