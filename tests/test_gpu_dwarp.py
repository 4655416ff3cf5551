"""The differentiable warp on the GPU against the oracle: forward values, the
hand-written backward (image and parameter gradients), a finite-difference
check of the GPU gradient, and the photometric descent of (t, phi, tx, ty)
toward a known ground truth.

Bars: forward |gpu - oracle| <= 1e-4 (values in [0, 1]: 1e-4 relative to full
scale; the fp32 geometry puts positions within ~1e-4 px and the image gradient
is below 0.5 per px); image gradient within 1e-4 of its largest magnitude;
parameter gradients within 2e-3 relative (fp32 sums of ~1e5 terms, atomics in
arbitrary order); GPU gradient vs fp64 central differences (step 1e-3) within
1e-2 relative.
"""
import ctypes as C
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_03479_gb300 import synth

pytestmark = pytest.mark.gpu

T_MAX = 5.7
K_FIX = math.ceil(4 * 0.8 * math.sqrt(T_MAX ** 2 - 1))


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


CASES = [  # (t0, phi0) of the fixed shape, then (t, phi, tx, ty)
    ((1.0, 0.0), (1.0, 0.0, 0.0, 0.0)),
    ((1.0, 0.0), (1.0137, 3.71, 0.43, -0.77)),
    ((2.0, 36.0), (2.1037, 33.3, 0.71, -0.43)),
    ((2.8284271247461903, 127.28), (2.91, 131.6, -3.2, 5.1)),
    ((5.656854249492381, 89.1), (5.44, 92.0, 7.5, -6.3)),
    # t far above the t the sizes were fixed for: whole view tiles map beyond
    # the canvas and read only its clamped last column
    ((1.4142135623730951, 101.8), (3.1, 101.8, 0.4, 0.0)),
]


def _setup(A, H=72, W=88):
    n = len(CASES)
    imgs = np.stack([synth.texture(H, W, 40 + i).astype(np.float64) / 255.0 for i in range(n)])
    lay = A.warp_layout(H, W, [c[0][0] for c in CASES], [c[0][1] for c in CASES], T_MAX)
    params = np.array([c[1] for c in CASES], np.float64)
    u = torch.from_numpy(imgs.astype(np.float32)).cuda()
    th = torch.from_numpy(params).cuda()
    ov = [O.dview(H, W, c[0][0], c[0][1], K_FIX, *c[1]) for c in CASES]
    return imgs, lay, u, th, ov


def test_forward_parity(A):
    ctx = A.Context()
    imgs, lay, u, th, ov = _setup(A)
    out = A.warp_forward(ctx, u, th, lay)
    torch.cuda.synchronize()
    for i, v in enumerate(ov):
        assert (lay.shapes[i].Wv, lay.shapes[i].Hv, lay.shapes[i].K) == (v.Wv, v.Hv, v.K)
        ref = O.dwarp_fwd(imgs[i].astype(np.float32).astype(np.float64), v)
        got = lay.view(out, i).cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-4, (i, np.abs(got - ref).max())
    # the identity case is exact
    assert np.array_equal(lay.view(out, 0).cpu().numpy(), imgs[0].astype(np.float32))


def test_backward_parity_and_finite_differences(A):
    ctx = A.Context()
    imgs, lay, u, th, ov = _setup(A)
    rng = np.random.default_rng(3)
    vbar = rng.standard_normal(lay.total).astype(np.float32)
    ub, pb = A.warp_backward(ctx, u, th, lay, torch.from_numpy(vbar).cuda())
    torch.cuda.synchronize()
    ub, pb = ub.cpu().numpy().astype(np.float64), pb.cpu().numpy()
    for i, v in enumerate(ov):
        s = lay.shapes[i]
        yb = vbar[lay.voff[i]: lay.voff[i] + s.Wv * s.Hv].reshape(s.Hv, s.Wv).astype(np.float64)
        u32 = imgs[i].astype(np.float32).astype(np.float64)
        rub, rpb = O.dwarp_vjp(u32, v, yb)
        assert np.abs(ub[i] - rub).max() <= 1e-4 * max(1.0, np.abs(rub).max()), i
        for k in range(4):
            assert abs(pb[i, k] - rpb[k]) <= 2e-3 * max(1.0, abs(rpb[k])), (i, k, pb[i, k], rpb[k])
        if i == 2:   # the GPU gradient against fp64 central differences, step 1e-3
            p0 = list(CASES[i][1])

            def f(p):
                return float((O.dwarp_fwd(u32, O.dview(72, 88, *CASES[i][0], K_FIX, *p)) * yb).sum())

            for k in range(4):
                a, b = list(p0), list(p0)
                a[k] += 1e-3
                b[k] -= 1e-3
                fd = (f(a) - f(b)) / 2e-3
                assert abs(pb[i, k] - fd) <= 1e-2 * max(1.0, abs(fd)), (k, pb[i, k], fd)


def test_autograd_function_matches_backward(A):
    ctx = A.Context()
    imgs, lay, u, th, ov = _setup(A)
    u = u.clone().requires_grad_(True)
    th = th.clone().requires_grad_(True)
    w = torch.randn(lay.total, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    out = A.WarpFunction.apply(u, th, ctx, lay)
    (out[: lay.total] * w).sum().backward()
    ub, pb = A.warp_backward(ctx, u.detach(), th.detach(), lay, w)
    assert torch.allclose(u.grad, ub, atol=1e-5, rtol=1e-4)
    assert torch.allclose(th.grad, pb, atol=1e-6, rtol=1e-4)


def _nearest_grid(t, phi):
    ts = np.sqrt(2.0) ** np.arange(6)
    k = int(np.argmin(np.abs(np.log(ts) - math.log(t))))
    if k == 0:
        return 1.0, 0.0
    step = 72.0 / ts[k]
    return float(ts[k]), float((round(phi / step) * step) % 180.0)


def test_photometric_descent_refines_tilt_and_rotation(A):
    """Ground truth (t*, phi*, tx*, ty*): t* ~ U[1.05, 5.7], phi* ~ U[0, 180),
    |tx*|, |ty*| <= 8 px; the start is the nearest view of the sampling grid
    (Sec. III-B) with no translation; 20 Adam steps on the L2 photometric loss
    against the target view rendered at the ground truth."""
    ctx = A.Context()
    rng = np.random.default_rng(4)
    n, H, W = 8, 192, 192
    imgs = np.stack([synth.texture(H, W, 900 + i).astype(np.float32) / 255.0 for i in range(n)])
    star = np.stack([rng.uniform(1.05, 5.7, n), rng.uniform(0, 180, n), rng.uniform(-8, 8, n),
                     rng.uniform(-8, 8, n)], 1)
    start = np.array([[*_nearest_grid(t, p), 0.0, 0.0] for t, p, _, _ in star])
    lay = A.warp_layout(H, W, start[:, 0], start[:, 1], T_MAX)
    u = torch.from_numpy(imgs).cuda()
    target = A.warp_forward(ctx, u, torch.from_numpy(star).cuda(), lay)
    hist, losses = A.refine(ctx, u, target, lay, torch.from_numpy(start).cuda(), steps=20,
                            lr=(0.1, 2.0, 1.0, 1.0))
    hist, losses = hist.cpu().numpy(), losses.cpu().numpy()
    e0 = np.abs(hist[0] - star)
    e1 = np.abs(hist[-1] - star)
    assert np.isfinite(losses).all()
    # every view's photometric loss goes down; most views converge (a start up
    # to 36/t degrees and 8 px away can sit in another basin of the texture)
    assert (losses[-1] < losses[0]).all(), losses[[0, -1]]
    assert np.median(losses[-1] / losses[0]) < 0.05, losses[[0, -1]]
    assert np.median(e1[:, 1] / np.maximum(e0[:, 1], 1e-9)) < 0.2       # rotation
    assert np.median(e1[:, 0] / np.maximum(e0[:, 0], 1e-9)) < 0.5       # tilt
    assert np.median(np.abs(e1[:, 2:]).max(1)) < 1.0                     # translation within a pixel


def test_loss_gradient_and_adam_step(A):
    """asift_warp_loss against numpy (fp32 squares, fp64 mean; the gradient
    2 d / count bit for bit), asift_warp_adam against the Adam update written
    out in fp64 (a view with a non-finite gradient takes a zero gradient, t
    clamped),
    and the parameter-only backward equal to the full one's parameter part."""
    ctx = A.Context()
    rng = np.random.default_rng(12)
    n, H, W = 5, 96, 96
    imgs = np.stack([synth.texture(H, W, 950 + i).astype(np.float32) / 255.0 for i in range(n)])
    th = np.stack([rng.uniform(1.2, 4.0, n), rng.uniform(0, 180, n), rng.uniform(-3, 3, n), rng.uniform(-3, 3, n)], 1)
    lay = A.warp_layout(H, W, th[:, 0], th[:, 1], 4.5)
    u = torch.from_numpy(imgs).cuda()
    tht = torch.from_numpy(th).cuda()
    v = A.warp_forward(ctx, u, tht, lay)
    tgt = A.warp_forward(ctx, u, tht + torch.tensor([0.05, 1.0, 0.3, -0.2], dtype=torch.float64, device="cuda"), lay)
    loss, vbar = A.warp_loss(ctx, v, tgt, lay)
    vh, th_, lh, gh = v.cpu().numpy(), tgt.cpu().numpy(), loss.cpu().numpy(), vbar.cpu().numpy()
    for i in range(n):
        o, cnt = int(lay.voff[i]), lay.shapes[i].Wv * lay.shapes[i].Hv
        d = vh[o:o + cnt] - th_[o:o + cnt]
        want = float(np.sum((d * d).astype(np.float64))) / cnt
        assert abs(lh[i] - want) <= 1e-9 * want + 1e-15, (i, lh[i], want)
        assert np.array_equal(gh[o:o + cnt], np.float32(2.0 / cnt) * d)
    # the parameter-only backward gives the full backward's parameter gradients
    ub, pb = A.warp_backward(ctx, u, tht, lay, vbar)
    none, pb2 = A.warp_backward(ctx, u, tht, lay, vbar, image_grad=False)
    assert none is None
    assert torch.allclose(pb, pb2, rtol=1e-6, atol=1e-9)
    # one Adam step
    g = pb2.clone()
    g[3, 1] = float("nan")                        # view 3 takes a zero gradient
    m0 = torch.from_numpy(rng.normal(0, 1e-3, (n, 4))).cuda()
    v0 = torch.from_numpy(rng.uniform(0, 1e-4, (n, 4))).cuda()
    p = tht.clone()
    p[0, 0] = 4.49                                # pushed past t_hi by the step below
    g[0, 0] = -50.0
    p0, gh, mh, vh0 = p.cpu().numpy(), g.cpu().numpy(), m0.cpu().numpy(), v0.cpu().numpy()
    m, vv = m0.clone(), v0.clone()
    lr = (C.c_double * 4)(0.1, 2.0, 1.0, 1.0)
    step, decay = 3, 0.88
    assert ctx.L.asift_warp_adam(ctx._ctx, n, C.c_void_p(p.data_ptr()), C.c_void_p(g.data_ptr()),
                                 C.c_void_p(m.data_ptr()), C.c_void_p(vv.data_ptr()), step, lr, decay, 1.0, 4.5,
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream)) == A.ASIFT_OK
    torch.cuda.synchronize()
    want = p0.copy()
    for i in range(n):
        gi = gh[i] if np.isfinite(gh[i]).all() else np.zeros(4)
        mi = 0.9 * mh[i] + 0.1 * gi
        vi = 0.999 * vh0[i] + 0.001 * gi * gi
        upd = decay ** step * np.array([0.1, 2.0, 1.0, 1.0]) * (mi / (1 - 0.9 ** (step + 1))) / \
            (np.sqrt(vi / (1 - 0.999 ** (step + 1))) + 1e-12)
        want[i] = p0[i] - upd
        want[i, 0] = min(max(want[i, 0], 1.0), 4.5)
    assert np.allclose(p.cpu().numpy(), want, rtol=1e-12, atol=1e-12)
    assert p[0, 0].item() == 4.5
