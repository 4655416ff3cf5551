"""Pins of the oracle's differentiable warp and its vector-Jacobian product.

The VJP is checked against the forward it transposes by two independent
routes: the adjoint identity <J x, y> = <x, J^T y> (the image part is linear),
and central finite differences of the forward in each parameter at generic
points (where every floor() is away from a switch, so the error is O(h^2)).
The forward itself is pinned to the ORB-path warp (same definition apart from
background and fixed K) and to exact identity / integer-shift cases.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_03479_gb300 import synth


def _img(h, w, seed):
    return synth.texture(h, w, seed).astype(np.float64) / 255.0


@pytest.mark.parametrize("t0,phi0,t,phi,tx,ty,K", [
    (2.0, 30.0, 2.1037, 33.3, 0.71, -0.43, 8),
    (1.4142135623730951, 101.8, 1.3771, 99.13, -1.27, 0.38, 6),
    (4.0, 162.0, 4.313, 158.77, 0.11, 2.33, 14),
    (1.0, 0.0, 1.0137, 3.71, 0.0, 0.0, 4),
])
def test_vjp_adjoint_and_finite_differences(t0, phi0, t, phi, tx, ty, K):
    rng = np.random.default_rng(7)
    u = _img(40, 52, 3)
    v = O.dview(40, 52, t0, phi0, K, t, phi, tx, ty)
    y = rng.standard_normal((v.Hv, v.Wv))
    ub, pb = O.dwarp_vjp(u, v, y)
    # adjoint identity in the image (linear part)
    x = rng.standard_normal(u.shape)
    lhs = float((O.dwarp_fwd(x, v) * y).sum())
    rhs = float((x * ub).sum())
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    # parameters: central differences, step 1e-4
    th = [t, phi, tx, ty]

    def f(p):
        vv = O.dview(40, 52, t0, phi0, K, *p)
        return float((O.dwarp_fwd(u, vv) * y).sum())

    for i in range(4):
        a, b = list(th), list(th)
        h = 1e-4
        a[i] += h
        b[i] -= h
        fd = (f(a) - f(b)) / (2 * h)
        assert abs(fd - pb[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, pb[i])


def test_identity_and_integer_shift_are_exact():
    u = _img(30, 40, 5)
    v = O.dview(30, 40, 1.0, 0.0, 6)
    assert np.array_equal(O.dwarp_fwd(u, v), u)
    v = O.dview(30, 40, 1.0, 0.0, 6, 1.0, 0.0, 3.0, -2.0)
    out = O.dwarp_fwd(u, v)
    # out(x, y) = u(x + 3, y - 2) where that source pixel exists
    assert np.array_equal(out[2:, :-3], u[:-2, 3:])


def test_forward_equals_the_view_warp_inside_the_footprint():
    """With no translation the differentiable forward is the ORB-path warp
    (the definition of Eq. (2)-(4)) wherever the zero background and the
    clamp-to-edge sampling agree, i.e. well inside the footprint."""
    u8 = synth.texture(90, 120, 9)
    u = u8.astype(np.float64)
    for (t0, phi0) in [(2.0, 36.0), (2.8284271247461903, 127.28), (1.4142135623730951, 50.91)]:
        ov = O.make_view(90, 120, t0, phi0)
        a = O.warp_view(u8, ov)
        v = O.dview(90, 120, t0, phi0, ov.K)
        b = O.dwarp_fwd(u, v)
        m = a.mask.astype(bool)
        inner = m.copy()
        r = int(np.ceil((ov.K + 6) / ov.t)) + 1
        for s in range(1, r + 1):
            inner[:, s:] &= m[:, :-s]
            inner[:, :-s] &= m[:, s:]
        inner[:4] = inner[-4:] = False
        inner &= np.roll(m, 4, 0) & np.roll(m, -4, 0)
        assert inner.sum() > 200
        # the ORB path rounds cos, sin and t to Q31: positions differ by at most
        # 2^-31 (|dx| + |dy|) < 1e-7 px, values by |grad| * 1e-7 < 2e-5
        assert np.abs(a.f64[inner] - b[inner]).max() < 2e-5


def test_sigma_term_vanishes_at_t_one():
    """At t = 1 the blur is the identity for any K (sigma = 0), and the t-gradient
    has no sigma contribution (dg/dsigma -> 0 faster than dsigma/dt grows)."""
    u = _img(24, 28, 11)
    v = O.dview(24, 28, 1.0, 0.0, 5, 1.0, 12.0, 0.3, 0.2)
    y = np.ones((v.Hv, v.Wv))
    _, pb = O.dwarp_vjp(u, v, y)
    assert np.isfinite(pb).all()
