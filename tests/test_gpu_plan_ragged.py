"""The batched plan on a ragged mix at the full ORB settings of the mixed-size
configuration: six pairs of uneven sizes (550..1719 wide, 384..1043 high,
absolute tilts 30-85 deg, synth.mixed_pair), views t = sqrt2^k for k <= 5
(43 per image), 8 pyramid levels and 1000 keypoints per view, run through
asift.Plan with the autotuner's choice of launch shapes.

Bars: every pair's accepted pairs bit-identical to match_pair on that pair
alone; for every pair, one sampled view of image 1 against the oracle (warp
within 3e-3 grey levels, mask exact, ORB keypoints and descriptors bit-exact
when the oracle is fed the GPU's own u8 view) and the view's slice of the
pooled descriptors equal to orb_extract's; 200 sampled queries of pool 1
against the whole pool 2 bit-exact against the oracle's brute force.
"""
import multiprocessing as mp

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_03479_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

WARP_TOL = 3e-3          # grey levels: the warp's error bound (outer bar of the configuration: 1e-4 * 255)
L_, N_, KMAX = 8, 1000, 5
SEED, INDICES = 3100, (0, 1, 2, 3, 5, 7)


def _gen(i):
    p = synth.mixed_pair(SEED, i)
    return p.img1, p.img2


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


@pytest.fixture(scope="module")
def pairs():
    with mp.get_context("spawn").Pool(len(INDICES)) as pool:
        return pool.map(_gen, INDICES)


def test_ragged_plan_full_orb_settings(A, pairs):
    ctx = A.Context(n_levels=L_, n_features=N_)
    imgs = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    shapes = {a.shape for a, _ in pairs} | {b.shape for _, b in pairs}
    assert len(shapes) == len(pairs)              # ragged: no two pairs alike
    plan = A.Plan(ctx, [a for a, _ in imgs], [b for _, b in imgs], kmax=KMAX)
    tuning = plan.autotune(reps=1)
    assert plan.tuning() == tuning
    plan.run()
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = [plan.pairs(i).tobytes() for i in range(len(pairs))]
    counts = plan.pool_counts()
    plan.close()

    pc = ctx.pair_cfg(kmax=KMAX)
    pat = O.pattern()
    rng = np.random.default_rng(11)
    for i, ((a, b), (ta, tb)) in enumerate(zip(pairs, imgs)):
        out, n, ws = ctx.match_pair(ta, tb, pc)
        torch.cuda.synchronize()
        assert ctx.read_status(ws) == 0
        assert ctx.pairs_host(out, n).tobytes() == got[i], i
        kp1, d1, kp2, d2, m = ctx.inspect_pair(a.shape, b.shape, pc, ws)
        assert (len(kp1), len(kp2)) == (counts[2 * i], counts[2 * i + 1])
        assert len(kp1) > 1000 and len(kp2) > 1000, (i, len(kp1), len(kp2))

        # one sampled view of image 1: warp, mask and ORB against the oracle
        views = A.view_table(*a.shape, KMAX)
        vi = int(rng.integers(1, len(views)))
        vo = ctx.views(ta, [views[vi]], with_f32=True)
        orb = ctx.orb_extract(vo)
        torch.cuda.synchronize()
        assert ctx.read_status(ctx.last_orb_ws) == 0
        rk, rd, vc, _ = orb.host()
        ov = O.view_table(*a.shape, KMAX)[vi]
        ref = O.warp_view(a, ov)
        f = vo.view(0, "f32").cpu().numpy().astype(np.float64)
        err = float(np.abs(f - ref.f64).max())
        print(f"pair {i} {a.shape[1]}x{a.shape[0]} view {vi} (t {views[vi].t:.2f}): warp worst {err:.3e}")
        assert err <= WARP_TOL, (i, vi, err)
        u8, mk = vo.view(0, "u8").cpu().numpy(), vo.view(0, "mask").cpu().numpy()
        assert np.array_equal(mk, ref.mask), (i, vi)
        r = O.orb_view(u8, mk, L_, N_, 20, pat)
        assert vc[0] == len(r.kps), (i, vi)
        for fld in ("x", "y", "level", "bin", "r25"):
            assert np.array_equal(rk[fld], r.kps[fld]), (i, vi, fld)
        assert np.array_equal(rd, r.desc), (i, vi)
        sel = kp1["view"] == vi
        assert np.array_equal(d1[sel], rd), (i, vi)

        # sampled queries against the whole train pool
        qs = np.sort(rng.choice(len(d1), size=200, replace=False))
        mref = O.match(d1[qs], d2, 4, 5)
        assert np.array_equal(m["best"][qs], mref.best), i
        assert np.array_equal(m["d1"][qs].astype(np.int32), mref.d1), i
        assert np.array_equal(m["d2"][qs].astype(np.int32), mref.d2), i
