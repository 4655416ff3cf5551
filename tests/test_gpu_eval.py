"""GPU parity of the evaluation of accepted pairs: duplicate removal in
original coordinates, the Eq. (5)-(6) precision count, RANSAC [28] and the
Eq. (7) inliers, through asift_eval_pairs against the oracle on the same
pairs and the same random numbers.

Bars: kept pairs, counts, the best hypothesis and the inlier mask bit-exact
(every decision is the fp64 one, one rounding per operation in the same
order; the GPU takes most of them in fp32 under a rigorous error bound); the
fitted homographies within 1e-9 relative.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_03479_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


def _random_h(rng):
    return np.array([[1 + rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-20, 20)],
                     [rng.uniform(-0.2, 0.2), 1 + rng.uniform(-0.2, 0.2), rng.uniform(-20, 20)],
                     [rng.uniform(-3e-4, 3e-4), rng.uniform(-3e-4, 3e-4), 1.0]])


def _apply_h(H, pts):
    p = np.c_[pts, np.ones(len(pts))] @ H.T
    return p[:, :2] / p[:, 2:]


def _synthetic_pairs(A, rng, n, frac_in=0.6, dup_frac=0.2):
    """Pairs under a known homography: inliers within 1 px, outliers 20-200 px
    off, and copies of earlier pairs jittered inside the same pixels."""
    H = _random_h(rng)
    n0 = max(1, int(n * (1 - dup_frac)))
    p1 = rng.uniform(0, 1000, size=(n0, 2))
    inl = rng.random(n0) < frac_in
    a = rng.uniform(0, 2 * np.pi, n0)
    off = np.where(inl[:, None], rng.uniform(-1, 1, size=(n0, 2)),
                   rng.uniform(20, 200, n0)[:, None] * np.c_[np.cos(a), np.sin(a)])
    p2 = _apply_h(H, p1) + off
    base = np.c_[p1, p2]
    base = np.floor(base) + 0.5 + rng.uniform(-0.3, 0.3, size=base.shape)   # pixel centres +- 0.3
    rows = [base]
    if n > n0:
        src = rng.integers(0, n0, n - n0)
        rows.append(base[src] + rng.uniform(-0.15, 0.15, size=(n - n0, 4)))
    allp = np.concatenate(rows)[rng.permutation(n)] if n > n0 else rows[0]
    pairs = np.zeros(n, A.PAIR_DTYPE)
    for k, f in enumerate(("x1", "y1", "x2", "y2")):
        pairs[f] = allp[:, k].astype(np.float32)
    pairs["q"] = np.arange(n)
    pairs["t"] = rng.integers(0, 1 << 20, n)
    return H, pairs


def _upload(A, pairs, cap=None):
    cap = len(pairs) if cap is None else cap
    buf = np.zeros(max(cap, 1), A.PAIR_DTYPE)
    buf[:len(pairs)] = pairs
    out = torch.from_numpy(buf.view(np.uint8).copy()).cuda()
    n = torch.tensor([len(pairs)], dtype=torch.int32, device="cuda")
    return out, n


def _rnd(rng, n_hyp):
    r = rng.integers(0, 2 ** 32, size=(n_hyp, 4), dtype=np.uint64).astype(np.uint32)
    return r, torch.from_numpy(r.view(np.int32).copy()).cuda()


def _check(A, ctx, pairs, H, rnd_np, rnd_t, cap=None, th_sq=3.0, rth_sq=9.0):
    out, n = _upload(A, pairs, cap)
    uq, inl, cnt, res = ctx.eval_pairs(out, n, H_true=H, th_sq=th_sq, rnd=rnd_t, ransac_th_sq=rth_sq, counts=True)
    torch.cuda.synchronize()
    r = ctx.eval_result(res)
    keep = O.dedup(pairs)
    kept = pairs[keep]
    assert r.status == 0
    assert r.n_pairs == len(pairs) and r.n_unique == len(kept)
    got = uq[: len(kept) * A.PAIR_DTYPE.itemsize].cpu().numpy().view(A.PAIR_DTYPE)
    assert got.tobytes() == kept.tobytes()
    if H is not None:
        assert r.r_num == O.precision_count(kept, H, th_sq)
    else:
        assert r.r_num == -1
    if rnd_np is None:
        assert r.best_hyp == -1 and r.n_inliers == 0
        return r, kept
    ref = O.ransac(kept, rnd_np, rth_sq)
    c = cnt.cpu().numpy()[: len(rnd_np)]
    assert np.array_equal(c, ref.counts)
    assert r.best_hyp == ref.best
    if ref.best >= 0:
        Hg = np.array(r.H)
        assert np.abs(Hg - ref.Hs[ref.best]).max() <= 1e-9 * np.abs(ref.Hs[ref.best]).max()
    m = inl.cpu().numpy()[: len(kept)].astype(bool)
    assert np.array_equal(m, ref.inlier)
    assert r.n_inliers == int(ref.inlier.sum())
    assert not inl.cpu().numpy()[len(kept):].any()
    return r, kept


@pytest.mark.parametrize("n,n_hyp,seed", [(10, 16, 1), (257, 64, 2), (3000, 512, 3), (20000, 1024, 4)])
def test_eval_synthetic_pairs(A, n, n_hyp, seed):
    ctx = A.Context()
    rng = np.random.default_rng(500 + seed)
    H, pairs = _synthetic_pairs(A, rng, n)
    rnd_np, rnd_t = _rnd(rng, n_hyp)
    r, kept = _check(A, ctx, pairs, H, rnd_np, rnd_t)
    assert len(kept) < n                      # duplicates were planted and removed
    if n >= 257:
        # RANSAC recovers the planted homography: about 60% of the kept pairs are inliers
        assert r.n_inliers >= 0.5 * r.n_unique
        q = rng.uniform(100, 900, size=(10, 2))
        assert np.abs(_apply_h(np.array(r.H).reshape(3, 3), q) - _apply_h(H, q)).max() < 3


def test_eval_edge_cases(A):
    ctx = A.Context()
    rng = np.random.default_rng(510)
    H, pairs = _synthetic_pairs(A, rng, 50, dup_frac=0.0)
    rnd_np, rnd_t = _rnd(rng, 8)
    # no pairs at all
    _check(A, ctx, pairs[:0], H, rnd_np, rnd_t, cap=16)
    # fewer than four pairs: nothing to fit
    r, _ = _check(A, ctx, pairs[:3], H, rnd_np, rnd_t, cap=8)
    assert r.best_hyp == -1
    # no hypotheses, no true homography
    _check(A, ctx, pairs, None, None, None)
    # the count word above the capacity is clamped to it
    out, n = _upload(A, pairs)
    n.fill_(10 ** 6)
    _, _, _, res = ctx.eval_pairs(out, n, H_true=H, rnd=rnd_t)
    torch.cuda.synchronize()
    assert ctx.eval_result(res).n_pairs == len(pairs)
    # every pair a copy of the first: one kept
    same = np.repeat(pairs[:1], 40)
    r, kept = _check(A, ctx, same, H, rnd_np, rnd_t)
    assert r.n_unique == 1 and r.best_hyp == -1


def test_eval_on_match_pair_output(A):
    """The accepted pairs of the 320x240 pair with its known affine map:
    duplicates, precision, RANSAC and inliers equal the oracle's on the GPU's
    own pairs."""
    ctx = A.Context(n_levels=4, n_features=500)
    p = synth.pair_affine_small()
    t1, t2 = torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()
    pc = ctx.pair_cfg(kmax=2)
    out, n, ws = ctx.match_pair(t1, t2, pc)
    torch.cuda.synchronize()
    pairs = ctx.pairs_host(out, n)
    rng = np.random.default_rng(520)
    rnd_np, rnd_t = _rnd(rng, 1024)
    r, kept = _check(A, ctx, pairs, p.H12, rnd_np, rnd_t)
    # the views of one image find some correspondences more than once
    assert r.n_unique <= r.n_pairs
    # Eq. (5): precision of the kept pairs, and the RANSAC inliers agree with it
    prec = r.r_num / r.n_unique
    assert prec > 0.5
    assert r.n_inliers >= 0.8 * r.r_num


def test_batched_evaluation_of_a_plan(A):
    """The evaluation of all pairs of a plan in one launch per stage equals the
    oracle's on each pair's accepted pairs (and so asift_eval_pairs')."""
    ctx = A.Context(n_levels=4, n_features=300)
    ps = [synth.pair_affine_small(seed=1100 + k, H=H, W=W) for k, (H, W) in enumerate(((240, 320), (200, 260),
                                                                                          (180, 300)))]
    imgs1 = [torch.from_numpy(p.img1).cuda() for p in ps]
    imgs2 = [torch.from_numpy(p.img2).cuda() for p in ps]
    plan = A.Plan(ctx, imgs1, imgs2, kmax=2)
    plan.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(530)
    rnd_np, rnd_t = _rnd(rng, 256)
    res = plan.evaluate(H_true=[p.H12 for p in ps], rnd=rnd_t)
    for i, p in enumerate(ps):
        pairs = plan.pairs(i)
        r = res[i]
        kept = pairs[O.dedup(pairs)]
        assert r.status == 0 and r.n_pairs == len(pairs) and r.n_unique == len(kept)
        uq, inl, cnt = plan.eval_outputs(i, r.n_unique)
        assert uq.tobytes() == kept.tobytes()
        assert r.r_num == O.precision_count(kept, p.H12, 3.0)
        ref = O.ransac(kept, rnd_np, 9.0)
        assert np.array_equal(cnt, ref.counts) and r.best_hyp == ref.best
        assert np.array_equal(inl, ref.inlier) and r.n_inliers == int(ref.inlier.sum())
        # and the single-pair entry point gives the same result
        out, n = _upload(A, pairs)
        _, _, _, res1 = ctx.eval_pairs(out, n, H_true=p.H12, rnd=rnd_t)
        r1 = ctx.eval_result(res1)
        assert (r1.n_unique, r1.r_num, r1.best_hyp, r1.n_inliers) == (r.n_unique, r.r_num, r.best_hyp, r.n_inliers)
    # no true homographies, no hypotheses
    res = plan.evaluate()
    assert all(r.r_num == -1 and r.best_hyp == -1 and r.n_inliers == 0 for r in res)
    plan.close()


def _scale_terms_abs(pairs):
    x1, y1 = pairs["x1"].astype(np.float64), pairs["y1"].astype(np.float64)
    x2, y2 = pairs["x2"].astype(np.float64), pairs["y2"].astype(np.float64)
    return float(np.abs(np.hypot(np.diff(x1), np.diff(y1)) - np.hypot(np.diff(x2), np.diff(y2))).sum())


@pytest.mark.parametrize("n,k", [(0, 1.0), (1, 1.0), (2, 0.5), (257, 0.8), (5000, 1.3)])
def test_scale_coefficient_parity(A, n, k):
    """Eq. (1) on the GPU against the oracle (fp64 on both sides, different
    summation orders: within 1e-9 of the sum of |terms|)."""
    ctx = A.Context()
    rng = np.random.default_rng(540 + n)
    p1 = rng.uniform(0, 900, size=(n, 2))
    th = 0.4
    R = k * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    p2 = p1 @ R.T + rng.normal(0, 0.5, size=(n, 2))
    pairs = np.zeros(n, A.PAIR_DTYPE)
    pairs["x1"], pairs["y1"], pairs["x2"], pairs["y2"] = p1[:, 0], p1[:, 1], p2[:, 0], p2[:, 1]
    pairs["d1"] = rng.integers(0, 100, n)
    out, cnt = _upload(A, pairs, cap=max(n, 4))
    f = float(ctx.scale_coefficient(out, cnt).item())
    ref = O.scale_coefficient(pairs)
    assert abs(f - ref) <= 1e-9 * _scale_terms_abs(pairs) + 1e-9, (f, ref)
    if n > 100:
        assert (f > 0) == (k < 1)


def test_base_image_selection_on_match_pair_outputs(A):
    """f1 and f2 on the accepted pairs of both matching directions equal the
    oracle's on the same pairs, and the image showing the scene larger (a
    1.6x magnified view of a texture, against the texture) is chosen as the
    reference (Sec. III-A)."""
    ctx = A.Context(n_levels=8, n_features=500)
    tex = synth.texture(240, 320, 77)
    big = np.ascontiguousarray(O.warp_view(tex, O.make_view(240, 320, 1.0, 0.0, 1.6)).u8)
    pc = ctx.pair_cfg(kmax=0)
    f = []
    for a, b in ((big, tex), (tex, big)):
        out, n, _ = ctx.match_pair(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), pc)
        fg = float(ctx.scale_coefficient(out, n).item())
        pairs = ctx.pairs_host(out, n)
        ref = O.scale_coefficient(pairs)
        assert abs(fg - ref) <= 1e-9 * _scale_terms_abs(pairs) + 1e-9
        f.append(fg)
    f1, f2, reference = ctx.base_image(torch.from_numpy(big).cuda(), torch.from_numpy(tex).cuda(), pc)
    assert (f1, f2) == (f[0], f[1])
    assert reference == 0 and f1 > 0 > f2
