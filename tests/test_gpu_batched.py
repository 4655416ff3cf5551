"""Batched form (one launch per stage over all views of many pairs, replayed
from a CUDA graph, launch shapes from the autotuner) against the per-pair
path: every pair's pools, matches and accepted pairs must be bit-identical to
match_pair on that pair alone (which is itself bit-exact against the oracle,
tests/test_gpu_parity.py), whatever the tuning, with or without the graph."""
import numpy as np
import pytest
import torch

from paper_2503_03479_gb300 import synth

pytestmark = pytest.mark.gpu

L_, N_, KMAX = 4, 200, 3


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


def _pairs():
    """Uneven sizes, including a flat image (no keypoints) and a tiny one."""
    shapes = [((150, 200), (260, 180)), ((240, 320), (240, 320)), ((211, 161), (157, 201)),
              ((96, 128), (100, 130)), ((60, 70), (180, 240))]
    out = []
    for i, (s1, s2) in enumerate(shapes):
        a = synth.texture(*s1, 500 + i)
        b = synth.texture(*s2, 600 + i)
        if i == 3:
            b = np.full(s2, 90, np.uint8)
        out.append((torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()))
    # one pair that really matches
    p = synth.pair_affine_small(seed=1005)
    out.append((torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()))
    return out


def _reference(A, ctx, pairs):
    ref = []
    pc = ctx.pair_cfg(kmax=KMAX)
    for a, b in pairs:
        out, n, ws = ctx.match_pair(a, b, pc)
        torch.cuda.synchronize()
        assert ctx.read_status(ws) == 0
        ref.append(ctx.pairs_host(out, n).tobytes())
    return ref


def test_batched_plan_equals_per_pair(A):
    ctx = A.Context(n_levels=L_, n_features=N_)
    pairs = _pairs()
    ref = _reference(A, ctx, pairs)
    assert sum(len(r) for r in ref) > 0
    plan = A.Plan(ctx, [p[0] for p in pairs], [p[1] for p in pairs], kmax=KMAX)
    for rep in range(2):                      # graph replays are repeatable
        plan.run()
        torch.cuda.synchronize()
        assert plan.status() == 0
        for i in range(len(pairs)):
            assert plan.pairs(i).tobytes() == ref[i], (rep, i)
    counts = plan.pool_counts()
    assert counts[7] == 0                     # the flat image has no keypoints
    plan.close()


def test_batched_plan_without_graph_and_with_tuning(A):
    ctx = A.Context(n_levels=L_, n_features=N_)
    pairs = _pairs()[:4]
    ref = _reference(A, ctx, pairs)
    plan = A.Plan(ctx, [p[0] for p in pairs], [p[1] for p in pairs], kmax=KMAX, use_graph=False,
                  tuning={"warp_grid": 152, "pyramid_grid": 300, "detect_grid": 152, "match_grid": 152,
                          "match_target_items": 77})
    plan.run()
    torch.cuda.synchronize()
    for i in range(len(pairs)):
        assert plan.pairs(i).tobytes() == ref[i], i
    plan.close()


def test_autotuner_picks_valid_shapes_and_keeps_results(A):
    ctx = A.Context(n_levels=L_, n_features=N_)
    pairs = _pairs()
    ref = _reference(A, ctx, pairs)
    plan = A.Plan(ctx, [p[0] for p in pairs], [p[1] for p in pairs], kmax=KMAX)
    t = plan.autotune(reps=2)
    assert set(t) == {"warp_grid", "pyramid_grid", "detect_grid", "match_grid", "match_target_items",
                      "match_engine", "warp_seg"}
    assert t["warp_seg"] in (0, 384, 512, 768)
    assert all(v >= 0 for v in t.values())
    # the tuner picks an engine explicitly when the device has tensor cores
    major, _ = torch.cuda.get_device_capability()
    assert t["match_engine"] in ((A.MATCH_CUDA_CORES, A.MATCH_TENSOR_CORES) if major == 10 else (0,))
    assert plan.tuning() == t
    plan.run()
    torch.cuda.synchronize()
    for i in range(len(pairs)):
        assert plan.pairs(i).tobytes() == ref[i], i
    plan.close()


def test_every_warp_tile_shape_gives_the_same_pairs(A):
    """The view simulation's tile shape (canvas columns per tile) is speed
    only: every shape the autotuner tries, and the widest, give the same
    accepted pairs, bit for bit."""
    ctx = A.Context(n_levels=L_, n_features=N_)
    pairs = _pairs()
    ref = _reference(A, ctx, pairs)
    plan = A.Plan(ctx, [p[0] for p in pairs], [p[1] for p in pairs], kmax=KMAX)
    base = plan.tuning()
    for seg in (64, 256, 384, 576, 768, 1024):
        plan.set_tuning(dict(base, warp_seg=seg))
        assert plan.tuning()["warp_seg"] == seg
        plan.run()
        torch.cuda.synchronize()
        assert plan.status() == 0
        for i in range(len(pairs)):
            assert plan.pairs(i).tobytes() == ref[i], (seg, i)
    with pytest.raises(A.AsiftError):
        plan.set_tuning(dict(base, warp_seg=32))
    plan.close()


def test_plan_rejects_bad_arguments(A):
    ctx = A.Context(n_levels=L_, n_features=N_)
    a = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AsiftError):
        A.Plan(ctx, [a], [a[:, :0]], kmax=KMAX)
