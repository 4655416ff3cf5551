"""GPU parity of the coarse stage (Sec. III-B): views carrying Eq. (2)'s scale
s = 1 + k ds, ORB on them, matching of the reference's parameter groups
against the unwarped target, and the per-view match counts with their argmax.

Bars: the warp within 3e-3 grey levels (its error bound; the configuration's
outer bar is 1e-4 of full scale); ORB, matches, counts and the argmax
bit-exact against the oracle fed the GPU's own u8 views and descriptor pools.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_03479_gb300 import synth

pytestmark = pytest.mark.gpu

WARP_TOL = 3e-3          # grey levels: the warp's error bound (outer bar of the configuration: 1e-4 * 255)


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


def _oracle_view(v):
    return O.make_view(v.H, v.W, v.t, v.phi_deg, scale=v.s)


def test_scaled_warp_parity(A):
    ctx = A.Context()
    img = synth.texture(101, 143, 31)
    views = A.view_table(101, 143, 3, 0.5) + [A.make_view(101, 143, 2.6, 33.0, s) for s in (1.25, 2.75, 4.0)]
    t = torch.from_numpy(img).cuda()
    vo = ctx.views(t, views, with_f32=True)
    torch.cuda.synchronize()
    for i, v in enumerate(views):
        ov = _oracle_view(v)
        assert (ov.Wr, ov.Hr, ov.Wv, ov.Hv, ov.cq, ov.sq, ov.tq, ov.K) == (v.Wr, v.Hr, v.Wv, v.Hv, v.cq, v.sq, v.tq, v.K)
        ref = O.warp_view(img, ov)
        f = vo.view(i, "f32").cpu().numpy().astype(np.float64)
        assert f.shape == ref.f64.shape
        assert np.abs(f - ref.f64).max() <= WARP_TOL, i
        assert np.array_equal(vo.view(i, "mask").cpu().numpy(), ref.mask), i
        du = np.abs(vo.view(i, "u8").cpu().numpy().astype(int) - ref.u8.astype(int))
        near_tie = np.abs(np.abs(ref.f64 - np.floor(ref.f64)) - 0.5) < 3e-3
        assert (du[~near_tie] == 0).all() and (du <= 1).all(), i


@pytest.mark.parametrize("H,W,kmax,ds", [(101, 143, 3, 0.5), (157, 201, 6, 0.0), (64, 80, 2, 1.0)])
def test_nearest_warp_parity(A, H, W, kmax, ds):
    """asift_views_nearest against the oracle's nearest-neighbour views: fp32
    within 3e-3 grey levels (the only rounding is the Gaussian's fp32 sum),
    the mask bit-exact, u8 equal except at rounding ties."""
    ctx = A.Context()
    img = synth.texture(H, W, 40 + kmax)
    views = A.view_table(H, W, kmax, ds) + [A.make_view(H, W, t, phi, s) for t, phi, s in
                                             ((1.0, 37.0, 1.0), (2.6, 33.0, 2.75), (7.9, 151.0, 1.0))]
    vo = ctx.views(torch.from_numpy(img).cuda(), views, with_f32=True, nearest=True)
    torch.cuda.synchronize()
    for i, v in enumerate(views):
        ref = O.warp_view_nn(img, _oracle_view(v))
        f = vo.view(i, "f32").cpu().numpy().astype(np.float64)
        assert f.shape == ref.f64.shape
        assert np.abs(f - ref.f64).max() <= WARP_TOL, i
        if v.K == 0:
            assert np.array_equal(f, ref.f64), i       # no arithmetic: the pixels themselves
        assert np.array_equal(vo.view(i, "mask").cpu().numpy(), ref.mask), i
        du = np.abs(vo.view(i, "u8").cpu().numpy().astype(int) - ref.u8.astype(int))
        near_tie = np.abs(np.abs(ref.f64 - np.floor(ref.f64)) - 0.5) < 3e-3
        assert (du[~near_tie] == 0).all() and (du <= 1).all(), i


def test_nearest_per_view_and_batched_forms_agree(A):
    ctx = A.Context(n_levels=4, n_features=300)
    p = synth.pair_affine_small(seed=1005)
    t1, t2 = torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()
    got = []
    for per_view in (False, True):
        pc = ctx.pair_cfg(kmax=2, per_view=per_view, coarse=True, nearest=True)
        out, n, ws = ctx.match_pair(t1, t2, pc)
        torch.cuda.synchronize()
        assert ctx.read_status(ws) == 0
        got.append(ctx.pairs_host(out, n).tobytes())
    assert got[0] == got[1] and len(got[0]) > 0


def test_scaled_orb_parity(A):
    L, N = 4, 300
    ctx = A.Context(n_levels=L, n_features=N)
    img = synth.texture(120, 160, 32)
    views = A.view_table(120, 160, 2, 0.5)
    vo = ctx.views(torch.from_numpy(img).cuda(), views)
    orb = ctx.orb_extract(vo)
    torch.cuda.synchronize()
    kp, desc, vc, _ = orb.host()
    pat = O.pattern()
    total = 0
    for i in range(len(views)):
        u = vo.view(i, "u8").cpu().numpy()
        m = vo.view(i, "mask").cpu().numpy()
        ref = O.orb_view(u, m, L, N, 20, pat)
        n = len(ref.kps)
        assert vc[i] == n
        for f in ("x", "y", "level", "bin", "r25"):
            assert np.array_equal(kp[total:total + n][f], ref.kps[f]), (i, f)
        assert np.array_equal(desc[total:total + n], ref.desc), i
        total += n
    assert total > 1000


def _coarse_run(A, ctx, img1, img2, kmax, ds, nearest=False):
    pc = ctx.pair_cfg(kmax=kmax, coarse=True, ds=ds, nearest=nearest)
    t1, t2 = torch.from_numpy(img1).cuda(), torch.from_numpy(img2).cuda()
    out, n, ws = ctx.match_pair(t1, t2, pc)
    counts, best = ctx.view_counts(img1.shape, img2.shape, pc, ws)
    torch.cuda.synchronize()
    assert ctx.read_status(ws) == 0
    return pc, ctx.pairs_host(out, n), ws, counts.cpu().numpy(), int(best.item())


@pytest.mark.parametrize("kmax,ds,nearest", [(2, 0.5, False), (3, 0.25, False), (0, 0.5, False), (2, 0.5, True),
                                             (3, 0.5, True)])
def test_coarse_counts_and_argmax_equal_oracle(A, kmax, ds, nearest):
    L, N = 4, 400
    ctx = A.Context(n_levels=L, n_features=N)
    p = synth.pair_affine_small(seed=1003)
    pc, pairs, ws, counts, best = _coarse_run(A, ctx, p.img1, p.img2, kmax, ds, nearest)
    views1 = A.view_table(*p.img1.shape, kmax, ds)
    assert len(counts) == len(views1)
    kp1, d1, kp2, d2, m = ctx.inspect_pair(p.img1.shape, p.img2.shape, pc, ws)
    # image 1's pool is the scaled views' ORB, image 2's the single identity view
    vo = ctx.views(torch.from_numpy(p.img1).cuda(), views1, nearest=nearest)
    rk1, rd1, _, _ = ctx.orb_extract(vo).host()
    assert np.array_equal(kp1, rk1) and np.array_equal(d1, rd1)
    assert (kp2["view"] == len(views1)).all()
    u2 = ctx.views(torch.from_numpy(p.img2).cuda(), A.view_table(*p.img2.shape, 0))
    torch.cuda.synchronize()
    assert np.array_equal(u2.view(0, "u8").cpu().numpy(), p.img2)
    ref2 = O.orb_view(p.img2, u2.view(0, "mask").cpu().numpy(), L, N, 20, O.pattern())
    for f in ("x", "y", "level", "bin", "r25"):
        assert np.array_equal(kp2[f], ref2.kps[f]), f
    assert np.array_equal(d2, ref2.desc)
    # matches, counts per view and the best parameter group
    ref = O.match(d1, d2, 4, 5)
    assert np.array_equal(m["best"], ref.best)
    acc = np.flatnonzero(ref.accepted)
    assert np.array_equal(pairs["q"], acc)
    want = np.bincount(kp1["view"][acc].astype(np.int64), minlength=len(views1))
    assert np.array_equal(counts, want)
    assert best == int(np.argmax(want))           # first maximum: the lowest view index
    # back-projection through the scaled views
    ov1 = O.view_table_scaled(*p.img1.shape, kmax, ds)
    for r in pairs[:: max(1, len(pairs) // 100)]:
        k1 = kp1[r["q"]]
        x1, y1 = O.backproject(ov1[k1["view"]], int(k1["level"]), float(k1["x"]), float(k1["y"]))
        assert abs(r["x1"] - x1) < 1e-3 and abs(r["y1"] - y1) < 1e-3


@pytest.mark.parametrize("nearest", [False, True])
def test_coarse_finds_the_simulated_view(A, nearest):
    """A target that is exactly one parameter group's simulated view of the
    reference (made by the oracle) draws the most matches to that group."""
    L, N, kmax, ds = 4, 400, 2, 0.5
    ctx = A.Context(n_levels=L, n_features=N)
    img1 = synth.texture(150, 190, 33)
    table = O.view_table_scaled(150, 190, kmax, ds)
    warp = O.warp_view_nn if nearest else O.warp_view
    for star in (3, 7):
        img2 = np.ascontiguousarray(warp(img1, table[star]).u8)
        _, pairs, _, counts, best = _coarse_run(A, ctx, img1, img2, kmax, ds, nearest)
        assert best == star, (star, counts.tolist())
        assert counts[star] > 2 * np.delete(counts, star).max()


def test_view_counts_rejects_short_output(A):
    ctx = A.Context(n_levels=3, n_features=100)
    p = synth.pair_affine_small(seed=1004, H=64, W=80)
    pc, _, ws, counts, _ = _coarse_run(A, ctx, p.img1, p.img2, 1, 0.5)
    short = torch.empty(len(counts) - 1, dtype=torch.int32, device="cuda")
    import ctypes as C
    rc = ctx.L.match_pair_view_counts(ctx._ctx, 64, 80, 64, 80, C.byref(pc), ws.data_ptr(), short.data_ptr(),
                                      short.numel(), None, None)
    assert rc == A.ASIFT_ERR_ARG
    pv = ctx.pair_cfg(kmax=1, per_view=True)
    rc = ctx.L.match_pair_view_counts(ctx._ctx, 64, 80, 64, 80, C.byref(pv), ws.data_ptr(), short.data_ptr(),
                                      short.numel(), None, None)
    assert rc == A.ASIFT_ERR_ARG


def test_batched_coarse_plan_equals_match_pair(A):
    """The coarse stage of several pairs of different sizes in one plan (one
    launch per stage, CUDA graph): every pair's accepted pairs, per-view counts
    and best group equal match_pair's on that pair alone."""
    ctx = A.Context(n_levels=4, n_features=300)
    rng = np.random.default_rng(600)
    imgs1, imgs2 = [], []
    for k, (H, W) in enumerate(((120, 160), (97, 131), (150, 190))):
        img1 = synth.texture(H, W, 610 + k)
        table = O.view_table_scaled(H, W, 2, 0.5)
        star = int(rng.integers(1, len(table)))
        imgs1.append(torch.from_numpy(img1).cuda())
        imgs2.append(torch.from_numpy(np.ascontiguousarray(O.warp_view_nn(img1, table[star]).u8)).cuda())
    plan = A.Plan(ctx, imgs1, imgs2, kmax=2, coarse=True, ds=0.5, nearest=True)
    plan.run()
    torch.cuda.synchronize()
    assert plan.status() == 0
    for i in range(len(imgs1)):
        pc = ctx.pair_cfg(kmax=2, coarse=True, ds=0.5, nearest=True)
        out, n, ws = ctx.match_pair(imgs1[i], imgs2[i], pc)
        c1, b1 = ctx.view_counts(tuple(imgs1[i].shape), tuple(imgs2[i].shape), pc, ws)
        c2, b2 = plan.view_counts(i)
        torch.cuda.synchronize()
        assert plan.pairs(i).tobytes() == ctx.pairs_host(out, n).tobytes()
        assert np.array_equal(c1.cpu().numpy(), c2.cpu().numpy()) and int(b1.item()) == int(b2.item())
    plan.close()
