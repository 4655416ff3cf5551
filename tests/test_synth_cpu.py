"""The texture generator's row-span shape rasteriser equals the plain
membership test applied to every pixel of each shape's bounding box (the
generator's definition), on several sizes and seeds.  The generator serves the
tests and the bench alike, so its output must not depend on how it is drawn."""
import math

import numpy as np
import pytest

from paper_2503_03479_gb300 import synth


def _ellipse_plain(img, rng):
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
    yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    dx, dy = xx - cx, yy - cy
    u = (dx * math.cos(th) + dy * math.sin(th)) / a
    v = (-dx * math.sin(th) + dy * math.cos(th)) / b
    img[y0:y1, x0:x1][u * u + v * v <= 1.0] = grey


def _polygon_plain(img, rng):
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
    yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    inside = np.ones(xx.shape, dtype=bool)
    for k in range(n):
        ax, ay = px[k], py[k]
        bx, by = px[(k + 1) % n], py[(k + 1) % n]
        inside &= (bx - ax) * (yy - ay) - (by - ay) * (xx - ax) >= 0
    img[y0:y1, x0:x1][inside] = grey


def _texture_plain(H, W, seed):
    rng = synth._rng(seed)
    noise = rng.standard_normal((H, W))
    F = np.fft.fft2(noise)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    F *= 1.0 / np.maximum(f, 1.0 / 64.0)
    img = np.real(np.fft.ifft2(F))
    img = (img - img.mean()) / (img.std() + 1e-12) * 40.0 + 128.0
    for _ in range(20 + (H * W) // 20000):
        if rng.uniform() < 0.5:
            _ellipse_plain(img, rng)
        else:
            _polygon_plain(img, rng)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


@pytest.mark.parametrize("H,W,seed", [(240, 320, 1000), (97, 131, 5), (31, 29, 9), (600, 500, 7), (768, 1024, 2000),
                                      (1080, 1920, 3)])
def test_row_span_rasteriser_equals_plain_membership_test(H, W, seed):
    assert np.array_equal(synth.texture(H, W, seed), _texture_plain(H, W, seed))
