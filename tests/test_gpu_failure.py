"""Failure detection on the device, without a GPU fault: capacity overflows
and a bounded wait that runs out end in a status word the host reads, and the
context stays usable for the next call.

  * output capacity: match_pair with room for fewer accepted pairs than it
    finds writes the true count and the first `cap` pairs, and sets
    ASIFT_ERR_CAPACITY;
  * candidate capacity: with the ASIFT_HOOK_CAND_CAP test hook every pyramid
    level holds 16 corners, far fewer than NMS keeps on a textured view:
    ASIFT_ERR_CAPACITY, and the next call without the hook is bit-identical
    to a clean run;
  * bounded waits: with the ASIFT_HOOK_MATCH_STALL test hook the tensor-core
    matcher's MMA warp waits on a barrier nothing arrives at, with a 10 ms
    limit: the launch records ASIFT_ERR_TIMEOUT and returns (its copies
    landed, its tensor memory freed), and the next launch, which allocates
    the same tensor memory, gives the oracle's matches.
"""
import time

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
def pair():
    p = synth.pair_affine_small(seed=1002)
    return p, torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()


def _clean_run(A, ctx, t1, t2, pc):
    out, n, ws = ctx.match_pair(t1, t2, pc)
    torch.cuda.synchronize()
    assert ctx.read_status(ws) == A.ASIFT_OK
    return ctx.pairs_host(out, n).tobytes(), int(n.item())


def test_output_capacity_overflow_writes_true_count(A, pair):
    _, t1, t2 = pair
    ctx = A.Context(n_levels=4, n_features=500)
    pc = ctx.pair_cfg(kmax=2)
    ref, n_ref = _clean_run(A, ctx, t1, t2, pc)
    assert n_ref > 50
    cap = 10
    out = torch.zeros(cap * A.PAIR_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    _, _, ws = ctx.match_pair(t1, t2, pc, out, n_out)
    torch.cuda.synchronize()
    assert ctx.read_status(ws) == A.ASIFT_ERR_CAPACITY
    assert int(n_out.item()) == n_ref                        # the true count
    got = out.cpu().numpy().view(A.PAIR_DTYPE)
    assert got.tobytes() == ref[: cap * A.PAIR_DTYPE.itemsize]
    assert _clean_run(A, ctx, t1, t2, pc) == (ref, n_ref)    # the next call is clean


def test_candidate_capacity_hook(A, pair):
    _, t1, t2 = pair
    ctx = A.Context(n_levels=4, n_features=500)
    pc = ctx.pair_cfg(kmax=2)
    ref = _clean_run(A, ctx, t1, t2, pc)
    ctx.set_test_hook(A.HOOK_CAND_CAP, 16)
    out, n, ws = ctx.match_pair(t1, t2, pc)
    torch.cuda.synchronize()
    assert ctx.read_status(ws) == A.ASIFT_ERR_CAPACITY
    # orb_extract reports it too
    vo = ctx.views(t1, A.view_table(*t1.shape, 1))
    ctx.orb_extract(vo)
    torch.cuda.synchronize()
    assert ctx.read_status(ctx.last_orb_ws) == A.ASIFT_ERR_CAPACITY
    ctx.set_test_hook(A.HOOK_CAND_CAP, 0)
    assert _clean_run(A, ctx, t1, t2, pc) == ref
    vo = ctx.views(t1, A.view_table(*t1.shape, 1))
    ctx.orb_extract(vo)
    torch.cuda.synchronize()
    assert ctx.read_status(ctx.last_orb_ws) == A.ASIFT_OK


def test_hooks_reject_bad_values(A):
    ctx = A.Context()
    for hook, v in ((A.HOOK_CAND_CAP, -1), (A.HOOK_MATCH_STALL, 5), (A.HOOK_MATCH_STALL, 5_000_000_000), (99, 1)):
        with pytest.raises(A.AsiftError):
            ctx.set_test_hook(hook, v)


def test_tensor_core_wait_times_out_and_recovers(A, pair):
    major, _ = torch.cuda.get_device_capability()
    if major != 10:
        pytest.skip("the tensor-core matcher needs compute capability 10.x")
    _, t1, t2 = pair
    ctx = A.Context(n_levels=4, n_features=500)
    ctx.set_match_engine(A.MATCH_TENSOR_CORES)
    q = torch.from_numpy(synth.random_descriptors(3000, 21)).cuda()
    t = torch.from_numpy(synth.random_descriptors(2500, 22)).cuda()
    ref = O.match(q.cpu().numpy(), t.cpu().numpy(), 4, 5)
    ws = ctx.workspace("hamming", ctx.L.hamming_workspace_size(3000, 2500))

    ctx.set_test_hook(A.HOOK_MATCH_STALL, 10_000_000)        # 10 ms
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.hamming_match(q, t)                                  # reads its outputs: synchronises
    elapsed = time.perf_counter() - t0
    assert ctx.read_status(ws) == A.ASIFT_ERR_TIMEOUT
    assert elapsed < 2.0, elapsed                            # the 10 ms limit, not the default 4 s

    ctx.set_test_hook(A.HOOK_MATCH_STALL, 0)
    best, d1, d2, acc, nacc = ctx.hamming_match(q, t)
    assert ctx.read_status(ws) == A.ASIFT_OK
    assert np.array_equal(best, ref.best) and np.array_equal(d1, ref.d1) and np.array_equal(d2, ref.d2)
    assert np.array_equal(acc, ref.accepted) and nacc == int(ref.accepted.sum())

    # the whole pair path: the timed-out matcher leaves the status word set,
    # the accepted-pair output writes only pairs with a train index in the
    # pool, and the next call is bit-identical to a clean run
    pc = ctx.pair_cfg(kmax=2)
    clean = _clean_run(A, ctx, t1, t2, pc)
    ctx.set_test_hook(A.HOOK_MATCH_STALL, 10_000_000)
    _, _, wsp = ctx.match_pair(t1, t2, pc)
    torch.cuda.synchronize()
    assert ctx.read_status(wsp) == A.ASIFT_ERR_TIMEOUT
    ctx.set_test_hook(A.HOOK_MATCH_STALL, 0)
    assert _clean_run(A, ctx, t1, t2, pc) == clean
