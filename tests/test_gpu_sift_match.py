"""GPU SIFT matching (asift_sift_match) against the oracle's matcher with the
decisions taken in fp32 in the same fixed order (oracle.sift_match_f32, itself
pinned against exact brute force and the fp64 matcher): nearest index, both
squared distances and the ratio-test decision bit-exact, on random and
exactly representable descriptors (ties included) of sizes that span several
64 x 64 tiles, train slices and ragged tails, on device-side counts, on empty
sets and on the GPU's own SIFT descriptors of an image pair.  The accepted
pairs feed Eq. (1) (Sec. III-A) as the paper defines it, on SIFT matches.
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


def _unit(rng, n):
    x = np.abs(rng.random((n, 128)))
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def _gpu(A, ctx, q, t, **kw):
    out, pairs, n_pairs = ctx.sift_match(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), **kw)
    torch.cuda.synchronize()
    assert ctx.read_status(ctx.last_sift_match_ws) == A.ASIFT_OK
    nq = q.shape[0] if kw.get("n_q") is None else int(kw["n_q"].item())
    return out[: nq * A.L2_MATCH_DTYPE.itemsize].cpu().numpy().view(A.L2_MATCH_DTYPE), pairs, n_pairs


def _same(m, ref):
    assert np.array_equal(m["best"], ref.best)
    assert np.array_equal(m["d1"].view(np.uint32), ref.d1.view(np.uint32))
    assert np.array_equal(m["d2"].view(np.uint32), ref.d2.view(np.uint32))


@pytest.mark.parametrize("nq,nt,seed", [(1, 1, 0), (5, 2, 1), (65, 129, 2), (700, 1300, 3), (3001, 2500, 4)])
def test_sift_match_bit_exact_random(A, nq, nt, seed):
    ctx = A.Context()
    rng = np.random.default_rng(700 + seed)
    q, t = _unit(rng, nq), _unit(rng, nt)
    for i in range(min(nq, nt, 40)):              # near copies: a range of ratios
        t[(7 * i) % nt] = np.abs(q[i] + rng.normal(0, 0.004 * (i + 1), 128)).astype(np.float32)
    m, _, _ = _gpu(A, ctx, q, t)
    ref = O.sift_match_f32(q, t, 0.8)
    _same(m, ref)
    r2 = np.float32(0.8 * 0.8)
    acc = (m["best"] >= 0) & (nt >= 2) & (m["d1"] < (r2 * m["d2"]).astype(np.float32))
    assert np.array_equal(acc, ref.accepted)


def test_sift_match_exact_values_and_ties(A):
    """Multiples of 1/64: every fp32 step exact; duplicated trains make ties
    (lowest index wins, d2 = d1)."""
    ctx = A.Context()
    rng = np.random.default_rng(710)
    q = (rng.integers(0, 17, (300, 128)) / 64).astype(np.float32)
    t = (rng.integers(0, 17, (333, 128)) / 64).astype(np.float32)
    t[100:150] = q[:50]
    t[200:250] = q[:50]
    m, _, _ = _gpu(A, ctx, q, t)
    ref = O.sift_match_f32(q, t, 0.8)
    _same(m, ref)
    assert (m["best"][:50] == np.arange(100, 150)).all() and (m["d2"][:50] == 0).all()


def test_sift_match_device_counts_and_empty_sets(A):
    ctx = A.Context()
    rng = np.random.default_rng(720)
    q, t = _unit(rng, 500), _unit(rng, 400)
    nq = torch.tensor([333], dtype=torch.int32, device="cuda")
    nt = torch.tensor([251], dtype=torch.int32, device="cuda")
    m, _, _ = _gpu(A, ctx, q, t, n_q=nq, n_t=nt)
    _same(m, O.sift_match_f32(q[:333], t[:251], 0.8))
    # no train descriptor, and a single one (no second nearest: never accepted)
    zero = torch.zeros(1, dtype=torch.int32, device="cuda")
    m, _, _ = _gpu(A, ctx, q, t, n_t=zero)
    assert (m["best"] == -1).all() and np.isinf(m["d1"]).all() and np.isinf(m["d2"]).all()
    m, _, _ = _gpu(A, ctx, q, t[:1])
    _same(m, O.sift_match_f32(q, t[:1], 0.8))
    assert np.isinf(m["d2"]).all()
    e = torch.zeros((0, 128), dtype=torch.float32, device="cuda")
    out, _, _ = ctx.sift_match(e, torch.from_numpy(t).cuda())
    torch.cuda.synchronize()
    with pytest.raises(A.AsiftError):
        ctx.sift_match(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), ratio=1.5)


def _sift(A, ctx, img):
    kp, desc, n = ctx.sift_raw(torch.from_numpy(img).cuda(), max_kp=4000)
    torch.cuda.synchronize()
    k = min(int(n.item()), 4000)
    return kp, desc, n, k


def test_sift_match_on_gpu_sift_and_eq1(A):
    """The GPU's SIFT of both images of a pair, matched on the GPU: results
    equal the oracle's fp32 matcher on the GPU's own descriptors; the accepted
    pairs (query order, keypoint coordinates, distances at integer-descriptor
    scale) equal those rebuilt on the host; Eq. (1) over them equals the
    oracle's; and the image showing the scene larger is the reference."""
    ctx = A.Context()
    tex = synth.texture(240, 320, 79)
    big = np.ascontiguousarray(O.warp_view(tex, O.make_view(240, 320, 1.0, 0.0, 1.6)).u8)
    f = []
    for a, b in ((big, tex), (tex, big)):
        kq, dq, nq, k1 = _sift(A, ctx, a)
        kt, dt, nt, k2 = _sift(A, ctx, b)
        assert k1 > 100 and k2 > 100
        out, pairs, n_pairs = ctx.sift_match(dq, dt, n_q=nq, n_t=nt, kq=kq, kt=kt)
        torch.cuda.synchronize()
        assert ctx.read_status(ctx.last_sift_match_ws) == A.ASIFT_OK
        m = out[: k1 * A.L2_MATCH_DTYPE.itemsize].cpu().numpy().view(A.L2_MATCH_DTYPE)
        hq, ht = dq[:k1].cpu().numpy(), dt[:k2].cpu().numpy()
        ref = O.sift_match_f32(hq, ht, 0.8)
        _same(m, ref)
        acc = np.flatnonzero(ref.accepted)
        npairs = int(n_pairs.item())
        assert npairs == len(acc) and npairs > 20
        p = pairs[: npairs * A.PAIR_DTYPE.itemsize].cpu().numpy().view(A.PAIR_DTYPE)
        k1h = kq[: k1 * A.SIFT_KP_DTYPE.itemsize].cpu().numpy().view(A.SIFT_KP_DTYPE)
        k2h = kt[: k2 * A.SIFT_KP_DTYPE.itemsize].cpu().numpy().view(A.SIFT_KP_DTYPE)
        assert np.array_equal(p["q"], acc) and np.array_equal(p["t"], ref.best[acc])
        assert np.array_equal(p["x1"], k1h["x"][acc]) and np.array_equal(p["y2"], k2h["y"][ref.best[acc]])
        des = np.rint(np.float32(512) * np.sqrt(ref.d1[acc])).astype(np.int64)
        assert np.array_equal(p["d1"].astype(np.int64), des)
        fg = float(ctx.scale_coefficient(pairs, n_pairs).item())
        fo = O.scale_coefficient(p)
        terms = np.abs(np.diff(np.c_[p["x1"], p["y1"]].astype(np.float64), axis=0)).sum() + \
            np.abs(np.diff(np.c_[p["x2"], p["y2"]].astype(np.float64), axis=0)).sum()
        assert abs(fg - fo) <= 1e-9 * terms + 1e-9, (fg, fo)
        f.append(fg)
    # Sec. III-A: image 1 (the magnified view) is the reference when f1 > f2
    assert f[0] > 0 > f[1]
