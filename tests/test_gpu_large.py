"""The large extreme-tilt configuration through the batched plan: pairs of
4096x3072 uint8, views t = sqrt2^k for k <= 6 (t up to 8, 63 views per image),
ORB with 8 levels and 2000 keypoints per view, about 126k x 126k descriptors
matched per pair.  Checked against the oracle on sampled views, one view's
ORB and sampled queries, and against per-pair match_pair bit for bit.

The pairs follow the 1024x768 pair's recipe at this size (synth.large_pair):
a 2x canonical texture seen by image 1 with absolute tilt t1 and by image 2
through a homography with local tilt t2 along the perpendicular direction, plus
N(0, 2^2) noise, t1 and t2 drawn from [2, 1/cos 83 deg].
"""
import multiprocessing as mp

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_03479_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

WARP_TOL = 3e-3          # grey levels: the warp's error bound (outer bar of the configuration: 1e-4 * 255)
L_, N_, KMAX = 8, 2000, 6
H_, W_ = 3072, 4096


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


def _pair(index):
    p = synth.large_pair(31, index, H_, W_)
    return p.img1, p.img2


def test_large_pairs_plan_sampled_parity(A):
    ctx = A.Context(n_levels=L_, n_features=N_)
    with mp.get_context("spawn").Pool(2) as pool:
        pairs = pool.map(_pair, [0, 1])
    imgs = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    plan = A.Plan(ctx, [a for a, _ in imgs], [b for _, b in imgs], kmax=KMAX)
    plan.run()
    torch.cuda.synchronize()
    assert plan.status() == 0
    cnt = plan.pool_counts()
    views = A.view_table(H_, W_, KMAX)
    assert len(views) == 63
    print("pooled descriptors per image:", cnt.tolist())
    assert (cnt > 10000).all(), cnt
    got = [plan.pairs(i) for i in range(len(pairs))]
    assert all(len(g) > 500 for g in got)
    plan.close()

    # the plan equals match_pair on the first pair, and match_pair's pools are checked below
    pc = ctx.pair_cfg(kmax=KMAX)
    out, n, ws = ctx.match_pair(imgs[0][0], imgs[0][1], pc)
    torch.cuda.synchronize()
    assert ctx.read_status(ws) == 0
    assert ctx.pairs_host(out, n).tobytes() == got[0].tobytes()
    kp1, d1, kp2, d2, m = ctx.inspect_pair((H_, W_), (H_, W_), pc, ws)
    assert len(kp1) == cnt[0] and len(kp2) == cnt[1]

    # warp and ORB of sampled views of image 1 against the oracle
    img1 = pairs[0][0]
    ov = O.view_table(H_, W_, KMAX)
    vsel = [0, 30, 62]                       # t = 1, t = 4, the largest tilt
    vo_views = [views[i] for i in vsel]
    from test_gpu_parity import _views_gpu
    vo = _views_gpu(A, ctx, img1, vo_views, with_f32=True)
    orb = ctx.orb_extract(vo)
    rk, rd, vc, voff = orb.host()
    pat = O.pattern()
    for j, i in enumerate(vsel):
        ref = O.warp_view(img1, ov[i])
        f = vo.view(j, "f32").cpu().numpy().astype(np.float64)
        assert np.abs(f - ref.f64).max() <= WARP_TOL, i
        u, mk = vo.view(j, "u8").cpu().numpy(), vo.view(j, "mask").cpu().numpy()
        assert np.array_equal(mk, ref.mask)
        if i == 62:
            r = O.orb_view(u, mk, L_, N_, 20, pat)
            sl = slice(voff[j], voff[j] + vc[j])
            assert vc[j] == len(r.kps)
            for fld in ("x", "y", "level", "bin", "r25"):
                assert np.array_equal(rk[sl][fld], r.kps[fld])
            assert np.array_equal(rd[sl], r.desc)
        # the same view inside the pair pool (canonical order: view-major)
        sel = kp1["view"] == i
        assert np.array_equal(d1[sel], rd[voff[j]: voff[j] + vc[j]])

    # sampled queries against the whole 2000 x 63 train pool
    rng = np.random.default_rng(1)
    qs = np.sort(rng.choice(len(d1), size=200, replace=False))
    ref = O.match(d1[qs], d2, 4, 5)
    assert np.array_equal(m["best"][qs], ref.best)
    assert np.array_equal(m["d1"][qs].astype(np.int32), ref.d1)
    assert np.array_equal(m["d2"][qs].astype(np.int32), ref.d2)
