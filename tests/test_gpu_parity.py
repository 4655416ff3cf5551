"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Bars:
  * warp: |gpu_f32 - oracle_f64| <= WARP_TOL = 3e-3 grey levels on every view.
    The outer bar, 1e-4 relative to the 8-bit full scale (0.0255), is the
    configuration's; 3e-3 is the kernel's own error bound.  The GPU evaluates
    a 36-tap normalised fp32 sum (the rotation) and one fused filter of 2K + 6
    taps (Gaussian and tilt); with sum |w| <= 1.25 per Lanczos axis, fp32 unit
    roundoff u = 2^-24 and weights within ~1e-6 relative, the forward error is
    at most 255 (gamma_12 S^2 + 2e-6 S) ~ 1e-3 for the rotation and 255
    gamma_(2K+6) S_h ~ 1.3e-3 for the filter at K = 18 (t = 5.66): below
    3e-3 up to K = 36 (t = 11); rounding errors add as a random walk, so the
    observed errors are several times smaller.  u8 equal except within 3e-3 of a rounding tie (then at most
    1 apart); mask bit-exact (its decisions are exact Q32 integer comparisons
    on both sides).
  * ORB keypoints, orientation bins, Harris responses and descriptors:
    bit-exact when the oracle is fed the GPU's own uint8 view and mask.
  * matching: bit-exact (integers).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_03479_gb300 import synth

pytestmark = pytest.mark.gpu

WARP_TOL = 3e-3          # grey levels (outer bar of the configuration: 1e-4 * 255)


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


def _views_gpu(A, ctx, img, views, with_f32=True):
    t = torch.from_numpy(img).cuda()
    vo = ctx.views(t, views, with_f32=with_f32)
    torch.cuda.synchronize()
    return vo


def _oracle_views(views):
    """The oracle's own descriptors for the same (t, phi) list."""
    return [O.make_view(v.H, v.W, v.t, v.phi_deg) for v in views]


def _check_warp(A, ctx, img, views):
    vo = _views_gpu(A, ctx, img, views)
    worst = 0.0
    for i, (v, ov) in enumerate(zip(views, _oracle_views(views))):
        assert (ov.Wv, ov.Hv, ov.cq, ov.sq, ov.tq, ov.K) == (v.Wv, v.Hv, v.cq, v.sq, v.tq, v.K)
        ref = O.warp_view(img, ov)
        f = vo.view(i, "f32").cpu().numpy().astype(np.float64)
        u = vo.view(i, "u8").cpu().numpy()
        m = vo.view(i, "mask").cpu().numpy()
        assert f.shape == ref.f64.shape
        d = np.abs(f - ref.f64)
        worst = max(worst, float(d.max()))
        assert d.max() <= WARP_TOL, (i, float(d.max()))
        assert np.array_equal(m, ref.mask), i
        near_tie = np.abs(np.abs(ref.f64 - np.floor(ref.f64)) - 0.5) < 3e-3
        du = np.abs(u.astype(int) - ref.u8.astype(int))
        assert (du[~near_tie] == 0).all(), i
        assert (du <= 1).all(), i
    print(f"warp worst |gpu - oracle| over {len(views)} views: {worst:.3e}")
    return vo, worst


def test_warp_parity_small_pair(A):
    ctx = A.Context(n_levels=4, n_features=500)
    p = synth.pair_affine_small()
    for img in (p.img1, p.img2):
        views = A.view_table(*img.shape, 2)
        _check_warp(A, ctx, img, views)


def test_warp_parity_ragged_sizes_and_all_tilts(A):
    ctx = A.Context()
    img = synth.texture(157, 201, 77)
    views = A.view_table(157, 201, 6)          # 63 views, t up to 8, ragged tiles
    _check_warp(A, ctx, img, views)


def test_warp_exact_special_views(A):
    ctx = A.Context()
    img = synth.random_u8((61, 95), 3)
    views = [A.make_view(61, 95, 1.0, phi) for phi in (0.0, 90.0, 180.0, 270.0)]
    vo = _views_gpu(A, ctx, img, views)
    for i, k in enumerate((0, -1, 2, 1)):
        f = vo.view(i, "f32").cpu().numpy()
        assert np.array_equal(f, np.rot90(img, k).astype(np.float32))
        assert np.array_equal(vo.view(i, "u8").cpu().numpy(), np.rot90(img, k))


def test_warp_arbitrary_tilt_and_rotation(A):
    ctx = A.Context()
    img = synth.texture(130, 170, 5)
    views = [A.make_view(130, 170, t, phi) for t, phi in ((1.37, 12.5), (3.3, 97.0), (7.9, 151.0), (11.0, 44.0))]
    _check_warp(A, ctx, img, views)


def _check_orb(A, ctx, vo, L, N):
    orb = ctx.orb_extract(vo)
    torch.cuda.synchronize()
    assert ctx.read_status(ctx.last_orb_ws) == 0
    kp, desc, vc, voff = orb.host()
    pat = O.pattern()
    total = 0
    for i, v in enumerate(vo.views):
        u = vo.view(i, "u8").cpu().numpy()
        m = vo.view(i, "mask").cpu().numpy()
        ref = O.orb_view(u, m, L, N, 20, pat)
        n = len(ref.kps)
        assert vc[i] == n, (i, vc[i], n)
        assert voff[i] == total
        g = kp[total:total + n]
        for f in ("x", "y", "level", "bin", "r25"):
            assert np.array_equal(g[f], ref.kps[f]), (i, f)
        assert (g["view"] == i).all()
        assert np.array_equal(desc[total:total + n], ref.desc), i
        total += n
    assert total == int(orb.total.item())
    return kp, desc


def test_orb_parity_small_pair(A):
    ctx = A.Context(n_levels=4, n_features=500)
    p = synth.pair_affine_small()
    for img in (p.img1, p.img2):
        vo = _views_gpu(A, ctx, img, A.view_table(*img.shape, 2), with_f32=False)
        kp, _ = _check_orb(A, ctx, vo, 4, 500)
        assert len(kp) > 2000


def test_orb_parity_general_masks(A):
    """Masks that are not the views' own: a footprint with holes (rows not
    intervals), one scaled to 255, one with mixed nonzero values, beside
    untouched footprints.  Views whose masks are 0/1 intervals per row take
    the row-hull path; the others the mask planes; all bit-exact."""
    ctx = A.Context(n_levels=5, n_features=400)
    img = synth.texture(300, 360, 17)
    vo = _views_gpu(A, ctx, img, A.view_table(300, 360, 3), with_f32=False)
    rng = np.random.default_rng(5)
    for i in range(len(vo.views)):
        m = vo.view(i, "mask")
        H, W = m.shape
        if i % 4 == 1:      # holes: several rows split into two or more runs
            for _ in range(6):
                y, x = int(rng.integers(0, H - 20)), int(rng.integers(0, W - 20))
                m[y:y + 20, x:x + int(rng.integers(3, 20))] = 0
        elif i % 4 == 2:    # a footprint of 255s
            m.mul_(255)
        elif i % 4 == 3:    # nonzero values 1 and 3 mixed
            sel = torch.from_numpy(rng.random((H, W)) < 0.3).to(m.device)
            m[sel & (m > 0)] = 3
    _check_orb(A, ctx, vo, 5, 400)


def test_orb_parity_ragged_many_levels(A):
    ctx = A.Context(n_levels=6, n_features=300)
    img = synth.texture(211, 263, 91)
    vo = _views_gpu(A, ctx, img, A.view_table(211, 263, 5), with_f32=False)
    _check_orb(A, ctx, vo, 6, 300)


def test_orb_tiny_and_flat_views_give_no_keypoints(A):
    ctx = A.Context(n_levels=3, n_features=100)
    img = np.full((40, 30), 128, np.uint8)
    vo = _views_gpu(A, ctx, img, A.view_table(40, 30, 2), with_f32=False)
    orb = ctx.orb_extract(vo)
    assert int(orb.total.item()) == 0
    img2 = synth.texture(24, 24, 1)
    vo = _views_gpu(A, ctx, img2, A.view_table(24, 24, 1), with_f32=False)
    assert int(ctx.orb_extract(vo).total.item()) == 0


@pytest.mark.parametrize("nq,nt,seed", [(1, 1, 0), (5, 2, 1), (513, 257, 2), (1000, 1537, 3), (4099, 3001, 4)])
def test_match_parity_random(A, nq, nt, seed):
    ctx = A.Context()
    q = synth.random_descriptors(nq, seed)
    t = synth.random_descriptors(nt, seed + 50)
    if nt > 10:
        t[7] = q[0]
        t[9] = q[0]                 # tie at distance 0
        t[8] = q[min(1, nq - 1)] ^ 1
    best, d1, d2, acc, nacc = ctx.hamming_match(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda())
    ref = O.match(q, t)
    assert np.array_equal(best, ref.best) and np.array_equal(d1, ref.d1)
    assert np.array_equal(d2, ref.d2) and np.array_equal(acc, ref.accepted)
    assert nacc == int(ref.accepted.sum())


def test_match_empty_sets(A):
    ctx = A.Context()
    q = torch.from_numpy(synth.random_descriptors(10, 1)).cuda()
    e = torch.zeros((0, 32), dtype=torch.uint8, device="cuda")
    best, d1, d2, acc, n = ctx.hamming_match(q, e)
    assert (best == -1).all() and (d1 == 257).all() and not acc.any() and n == 0
    best, *_ , n = ctx.hamming_match(e, q)
    assert len(best) == 0 and n == 0


def _pair_pools_oracle(A, ctx, img, kmax, L, N):
    vo = _views_gpu(A, ctx, img, A.view_table(*img.shape, kmax), with_f32=False)
    orb = ctx.orb_extract(vo)
    kp, desc, _, _ = orb.host()
    return kp, desc


def test_match_pair_small_end_to_end(A):
    L, N, kmax = 4, 500, 2
    ctx = A.Context(n_levels=L, n_features=N)
    p = synth.pair_affine_small()
    t1, t2 = torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()
    outs = {}
    for per_view in (False, True):
        pc = ctx.pair_cfg(kmax=kmax, per_view=per_view)
        out, n, ws = ctx.match_pair(t1, t2, pc)
        torch.cuda.synchronize()
        assert ctx.read_status(ws) == 0
        pairs = ctx.pairs_host(out, n)
        kp1, d1, kp2, d2, m = ctx.inspect_pair(p.img1.shape, p.img2.shape, pc, ws)
        outs[per_view] = (pairs.tobytes(), kp1.tobytes(), d1.tobytes(), kp2.tobytes(), d2.tobytes(), m.tobytes())
    # the plain per-view launch sequence and the batched one agree bit for bit
    assert outs[False] == outs[True]
    pc = ctx.pair_cfg(kmax=kmax)
    out, n, ws = ctx.match_pair(t1, t2, pc)
    pairs = ctx.pairs_host(out, n)
    kp1, d1, kp2, d2, m = ctx.inspect_pair(p.img1.shape, p.img2.shape, pc, ws)
    # pools equal asift_views -> orb_extract (bit-exact vs the oracle elsewhere)
    rk1, rd1 = _pair_pools_oracle(A, ctx, p.img1, kmax, L, N)
    rk2, rd2 = _pair_pools_oracle(A, ctx, p.img2, kmax, L, N)
    nv1 = len(A.view_table(*p.img1.shape, kmax))
    rk2 = rk2.copy()
    rk2["view"] += nv1
    assert np.array_equal(kp1, rk1) and np.array_equal(d1, rd1)
    assert np.array_equal(kp2, rk2) and np.array_equal(d2, rd2)
    # matches equal the oracle's brute force on the GPU's descriptors
    ref = O.match(d1, d2, 4, 5)
    assert np.array_equal(m["best"], ref.best)
    assert np.array_equal(m["d1"].astype(np.int32), ref.d1) and np.array_equal(m["d2"].astype(np.int32), ref.d2)
    acc = np.flatnonzero(ref.accepted)
    assert np.array_equal(pairs["q"], acc) and np.array_equal(pairs["t"], ref.best[acc])
    # back-projection equals the oracle's (fp64 on both sides, fp32 output)
    v1 = O.view_table(*p.img1.shape, kmax)
    v2 = O.view_table(*p.img2.shape, kmax)
    for r in pairs[:: max(1, len(pairs) // 200)]:
        k1, k2 = kp1[r["q"]], kp2[r["t"]]
        x1, y1 = O.backproject(v1[k1["view"]], int(k1["level"]), float(k1["x"]), float(k1["y"]))
        x2, y2 = O.backproject(v2[k2["view"] - nv1], int(k2["level"]), float(k2["x"]), float(k2["y"]))
        assert abs(r["x1"] - x1) < 1e-3 and abs(r["y1"] - y1) < 1e-3
        assert abs(r["x2"] - x2) < 1e-3 and abs(r["y2"] - y2) < 1e-3
    # and the geometry is right: reprojection with the known affine (Eq. (5)-(6))
    x1 = np.c_[pairs["x1"], pairs["y1"], np.ones(len(pairs))] @ p.H12.T
    err = np.hypot(x1[:, 0] / x1[:, 2] - pairs["x2"], x1[:, 1] / x1[:, 2] - pairs["y2"])
    assert len(pairs) > 100 and np.median(err) < 1.5 and (err <= math.sqrt(3)).mean() >= 0.5


def test_match_pair_is_deterministic(A):
    ctx = A.Context(n_levels=4, n_features=500)
    p = synth.pair_affine_small(seed=1001)
    t1, t2 = torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()
    pc = ctx.pair_cfg(kmax=2)
    a = ctx.pairs_host(*ctx.match_pair(t1, t2, pc)[:2]).tobytes()
    b = ctx.pairs_host(*ctx.match_pair(t1, t2, pc)[:2]).tobytes()
    assert a == b and len(a) > 0


@pytest.mark.slow
def test_full_size_pair_sampled_parity(A):
    """1024x768 pair, 43 views per image, 8 levels, 1000 keypoints per view, in
    the launch configuration the bench times (one launch per stage over all
    views of both images).  Checked against the oracle on sampled views and
    sampled queries."""
    L, N, kmax = 8, 1000, 5
    ctx = A.Context(n_levels=L, n_features=N)
    p = synth.pair_extreme_tilt()
    t1, t2 = torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()
    pc = ctx.pair_cfg(kmax=kmax)
    out, n, ws = ctx.match_pair(t1, t2, pc)
    torch.cuda.synchronize()
    assert ctx.read_status(ws) == 0
    pairs = ctx.pairs_host(out, n)
    kp1, d1, kp2, d2, m = ctx.inspect_pair(p.img1.shape, p.img2.shape, pc, ws)
    assert len(kp1) > 10000 and len(kp2) > 10000
    # views and ORB on sampled views of image 1 (one per tilt), against the oracle
    views = A.view_table(*p.img1.shape, kmax)
    vo = _views_gpu(A, ctx, p.img1, views, with_f32=True)
    orb = ctx.orb_extract(vo)
    rk1, rd1, vc, voff = orb.host()
    assert np.array_equal(kp1, rk1) and np.array_equal(d1, rd1)
    ov = O.view_table(*p.img1.shape, kmax)
    pat = O.pattern()
    for i in (0, 2, 7, 20, 42):
        ref = O.warp_view(p.img1, ov[i])
        f = vo.view(i, "f32").cpu().numpy().astype(np.float64)
        err = float(np.abs(f - ref.f64).max())
        print(f"warp worst |gpu - oracle| on view {i} of the 1024x768 pair: {err:.3e}")
        assert err <= WARP_TOL, (i, err)
        u, mk = vo.view(i, "u8").cpu().numpy(), vo.view(i, "mask").cpu().numpy()
        assert np.array_equal(mk, ref.mask)
        r = O.orb_view(u, mk, L, N, 20, pat)
        sl = slice(voff[i], voff[i] + vc[i])
        assert vc[i] == len(r.kps)
        for fld in ("x", "y", "level", "bin", "r25"):
            assert np.array_equal(rk1[sl][fld], r.kps[fld])
        assert np.array_equal(rd1[sl], r.desc)
    # sampled queries against the whole train pool
    rng = np.random.default_rng(0)
    qs = np.sort(rng.choice(len(d1), size=300, replace=False))
    ref = O.match(d1[qs], d2, 4, 5)
    assert np.array_equal(m["best"][qs], ref.best)
    assert np.array_equal(m["d1"][qs].astype(np.int32), ref.d1)
    assert np.array_equal(m["d2"][qs].astype(np.int32), ref.d2)
    acc = (5 * m["d1"].astype(int) < 4 * m["d2"].astype(int))
    assert np.array_equal(pairs["q"], np.flatnonzero(acc))
    # reprojection sanity with the known homography: at a transition tilt near
    # 85 degrees most ratio-test survivors are wrong (no RANSAC here), but a
    # consistent set lands within 3 px (the oracle finds 62 of 1545 on this pair)
    x1 = np.c_[pairs["x1"], pairs["y1"], np.ones(len(pairs))] @ p.H12.T
    err = np.hypot(x1[:, 0] / x1[:, 2] - pairs["x2"], x1[:, 1] / x1[:, 2] - pairs["y2"])
    assert len(pairs) > 500 and (err <= 3.0).sum() >= 30
