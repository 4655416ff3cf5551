"""The two matcher engines (CUDA-core popcount scan, tensor-core +-1 fp8 matrix
product) against the oracle's brute force and against each other.

Both must give the oracle's result bit for bit: nearest index (lowest on
ties), d1, d2, the ratio-test decision and the accepted count.  Sizes span
several 256-query items and 128-train tiles with ragged tails on both sides;
special cases: exact duplicates (distance 0 ties), complements (distance 256),
all-equal pools (every distance tied), counts read from the device below the
capacities, and fewer than two trains.
"""
import ctypes as C

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


@pytest.fixture(scope="module")
def ctxs(A):
    out = {}
    for eng in (A.MATCH_CUDA_CORES, A.MATCH_TENSOR_CORES):
        c = A.Context()
        c.set_match_engine(eng)
        assert c.match_engine == eng
        out[eng] = c
    return out


def _run(A, ctx, q, t, num=4, den=5):
    r = ctx.hamming_match(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), num, den)
    torch.cuda.synchronize()
    ws = ctx._ws["hamming"]
    assert ctx.read_status(ws) == 0
    return r


def _assert_oracle(r, ref):
    best, d1, d2, acc, nacc = r
    assert np.array_equal(best, ref.best)
    assert np.array_equal(d1, ref.d1) and np.array_equal(d2, ref.d2)
    assert np.array_equal(acc, ref.accepted) and nacc == int(ref.accepted.sum())


def test_default_engine_is_tensor_cores_on_this_device(A):
    major, _ = torch.cuda.get_device_capability()
    ctx = A.Context()
    assert ctx.match_engine == (A.MATCH_TENSOR_CORES if major == 10 else A.MATCH_CUDA_CORES)


@pytest.mark.parametrize("nq,nt,seed", [
    (1, 1, 0), (1, 2, 1), (2, 129, 2), (255, 127, 3), (256, 128, 4), (257, 129, 5),
    (511, 1000, 6), (1000, 4097, 7), (3001, 2049, 8), (4099, 5003, 9),
])
def test_engines_equal_oracle_random(A, ctxs, nq, nt, seed):
    q = synth.random_descriptors(nq, seed)
    t = synth.random_descriptors(nt, seed + 100)
    if nt > 200:
        t[130] = q[0]                     # distance 0 twice: the lower index wins
        t[190] = q[0]
        t[150] = q[nq - 1] ^ 0xFF         # the complement: distance 256
        t[nt - 1] = q[nq // 2]            # in the ragged last tile
    ref = O.match(q, t)
    for eng, ctx in ctxs.items():
        _assert_oracle(_run(A, ctx, q, t), ref)


def test_engines_all_distances_tied(A, ctxs):
    """Every train equal: d1 = d2 for all queries, best = 0, nothing accepted."""
    q = synth.random_descriptors(700, 11)
    t = np.repeat(synth.random_descriptors(1, 12), 900, axis=0)
    ref = O.match(q, t)
    assert (ref.best == 0).all() and (ref.d1 == ref.d2).all()
    for ctx in ctxs.values():
        _assert_oracle(_run(A, ctx, q, t), ref)


def test_engines_few_distinct_trains(A, ctxs):
    """Trains drawn from 5 distinct descriptors (heavy ties at every distance)
    and queries near them: ties broken by the lowest index in every tile."""
    rng = np.random.default_rng(13)
    base = synth.random_descriptors(5, 14)
    t = base[rng.integers(0, 5, 2000)]
    q = base[rng.integers(0, 5, 600)].copy()
    flip = rng.integers(0, 256, 600)
    q[np.arange(600), flip >> 3] ^= (1 << (flip & 7)).astype(np.uint8)
    ref = O.match(q, t)
    for ctx in ctxs.values():
        _assert_oracle(_run(A, ctx, q, t), ref)


@pytest.mark.parametrize("num,den", [(4, 5), (1, 1), (0, 1), (7, 10)])
def test_engines_ratio_variants(A, ctxs, num, den):
    q = synth.random_descriptors(300, 21)
    t = synth.random_descriptors(700, 22)
    t[:300:3] = q[:300:3] ^ 3
    ref = O.match(q, t, num, den)
    for ctx in ctxs.values():
        _assert_oracle(_run(A, ctx, q, t, num, den), ref)


def test_engines_device_counts_below_capacity(A, ctxs):
    """Counts read from the device: only the first nq / nt rows take part; the
    rows past them hold garbage that must not leak into any result."""
    nq_cap, nt_cap, nq, nt = 900, 1300, 611, 1001
    q = synth.random_descriptors(nq_cap, 31)
    t = synth.random_descriptors(nt_cap, 32)
    t[nt:] = q[0]                          # would be a perfect match if it leaked
    ref = O.match(q[:nq], t[:nt])
    for ctx in ctxs.values():
        L = ctx.L
        dq, dt = torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda()
        cnt = torch.tensor([nq, nt], dtype=torch.int32, device="cuda")
        out = torch.full((nq_cap * 8,), 0xAB, dtype=torch.uint8, device="cuda")
        acc = torch.zeros(nq_cap, dtype=torch.uint8, device="cuda")
        nacc = torch.zeros(1, dtype=torch.int32, device="cuda")
        ws = torch.zeros(L.hamming_workspace_size(nq_cap, nt_cap), dtype=torch.uint8, device="cuda")
        rc = L.hamming_match(ctx._ctx, C.c_void_p(dq.data_ptr()), nq_cap, C.c_void_p(cnt.data_ptr()),
                             C.c_void_p(dt.data_ptr()), nt_cap, C.c_void_p(cnt.data_ptr() + 4), 4, 5,
                             C.c_void_p(out.data_ptr()), C.c_void_p(acc.data_ptr()), C.c_void_p(nacc.data_ptr()),
                             C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert ctx.read_status(ws) == 0
        m = out[: nq * 8].cpu().numpy().view(A.MATCH_DTYPE)
        assert np.array_equal(m["best"], ref.best)
        assert np.array_equal(m["d1"].astype(np.int32), ref.d1)
        assert np.array_equal(m["d2"].astype(np.int32), ref.d2)
        assert np.array_equal(acc[:nq].cpu().numpy().astype(bool), ref.accepted)
        assert int(nacc.item()) == int(ref.accepted.sum())
        # rows past the device count are left untouched
        assert (out[nq * 8:].cpu().numpy() == 0xAB).all()


def test_match_pair_engines_identical(A):
    p = synth.pair_affine_small(seed=77)
    t1, t2 = torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()
    res = {}
    for eng in (A.MATCH_CUDA_CORES, A.MATCH_TENSOR_CORES):
        ctx = A.Context(n_levels=4, n_features=500)
        ctx.set_match_engine(eng)
        pc = ctx.pair_cfg(kmax=3)
        out, n, ws = ctx.match_pair(t1, t2, pc)
        torch.cuda.synchronize()
        assert ctx.read_status(ws) == 0
        kp1, d1, kp2, d2, m = ctx.inspect_pair(p.img1.shape, p.img2.shape, pc, ws)
        res[eng] = (ctx.pairs_host(out, n).tobytes(), m.tobytes())
        ref = O.match(d1, d2, 4, 5)
        assert np.array_equal(m["best"], ref.best)
        assert np.array_equal(m["d2"].astype(np.int32), ref.d2)
    assert res[A.MATCH_CUDA_CORES] == res[A.MATCH_TENSOR_CORES]


def test_plan_engines_and_target_items_identical(A):
    """The batched plan over uneven pairs: both engines and several slicings
    (items per launch) give the same pairs bit for bit."""
    ctx = A.Context(n_levels=4, n_features=300)
    pairs = [synth.mixed_pair(5, i, wmin=320, wmax=720, hmin=240, hmax=540) for i in range(3)]
    imgs = [(torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()) for p in pairs]
    ref = None
    for tuning in ({"match_engine": A.MATCH_CUDA_CORES}, {"match_engine": A.MATCH_TENSOR_CORES},
                   {"match_engine": A.MATCH_TENSOR_CORES, "match_target_items": 1},
                   {"match_engine": A.MATCH_TENSOR_CORES, "match_target_items": 5000},
                   {"match_engine": A.MATCH_TENSOR_CORES, "match_grid": 7}):
        plan = A.Plan(ctx, [a for a, _ in imgs], [b for _, b in imgs], kmax=2, tuning=tuning)
        plan.run()
        torch.cuda.synchronize()
        assert plan.status() == 0
        got = [plan.pairs(i).tobytes() for i in range(len(pairs))]
        if ref is None:
            ref = got
            assert all(len(g) > 0 for g in got)
        assert got == ref, tuning
        plan.close()


def test_engine_argument_checks(A):
    ctx = A.Context()
    with pytest.raises(A.AsiftError):
        ctx.set_match_engine(3)
    with pytest.raises(A.AsiftError):
        ctx.set_match_engine(-1)


def test_workspace_alignment_checked(A):
    """Workspaces are 256-byte aligned; an offset one is an argument error
    (nothing enqueued), for match_pair and asift_views alike."""
    import ctypes as C
    ctx = A.Context(n_levels=4, n_features=200)
    img = torch.zeros((96, 128), dtype=torch.uint8, device="cuda")
    pc = ctx.pair_cfg(kmax=1)
    ws = ctx.match_pair_workspace((96, 128), (96, 128), pc)
    big = torch.zeros(ws.numel() + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AsiftError):
        ctx.match_pair(img, img, pc, ws=big[16:16 + ws.numel()])
    ctx.match_pair(img, img, pc, ws=big[256:256 + ws.numel()])
    torch.cuda.synchronize()
    views = A.view_table(96, 128, 1)
    nb = ctx.L.asift_views_workspace_size(96, 128, len(views))
    wsv = torch.zeros(nb + 256, dtype=torch.uint8, device="cuda")
    offs, total = A.view_offsets(views)
    u8 = torch.empty(total, dtype=torch.uint8, device="cuda")
    mask = torch.empty_like(u8)
    arr = A._view_array(views)
    for off, ok in ((16, False), (256, True)):
        st = ctx.L.asift_views(ctx._ctx, A._ptr(img), 96, 128, 128, arr, len(views), offs.ctypes.data_as(C.c_void_p),
                               None, A._ptr(u8), A._ptr(mask), C.c_void_p(wsv.data_ptr() + off), nb, A._stream())
        assert (st == 0) == ok, (off, st)
    torch.cuda.synchronize()
