"""match_pair keeps the host tables of its last few distinct calls (keyed by
every argument that shapes them).  Repeated calls, calls that evict entries,
and new image content in the same buffers must all give what a fresh context
gives for the same images."""
import numpy as np
import pytest
import torch

from paper_2503_03479_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(96, 128), (120, 160), (100, 150), (64, 200), (150, 90)]   # five keys, four cache entries


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


def _pair(shape, seed):
    H, W = shape
    img1 = synth.texture(H, W, seed)
    A2 = synth.tilt_about_centre((H, W), (H, W), 1.6, 30.0 + seed % 50, 1.0)
    img2 = np.clip(np.rint(synth.render(img1, A2, (H, W), ss=1)), 0, 255).astype(np.uint8)
    return img1, img2


def _fresh(A, img1, img2):
    ctx = A.Context(n_levels=4, n_features=300)
    pc = ctx.pair_cfg(kmax=2)
    out, n, _ = ctx.match_pair(torch.from_numpy(img1).cuda(), torch.from_numpy(img2).cuda(), pc)
    return ctx.pairs_host(out, n).tobytes()


def test_repeated_evicted_and_refilled_calls_match_fresh_contexts(A):
    pairs = [_pair(s, 40 + i) for i, s in enumerate(SHAPES)]
    ref = [_fresh(A, a, b) for a, b in pairs]
    assert all(len(r) > 0 for r in ref)
    ctx = A.Context(n_levels=4, n_features=300)
    pc = ctx.pair_cfg(kmax=2)
    big = max(int(ctx.match_pair_workspace(s, s, pc).numel()) for s in SHAPES)
    ws = torch.zeros(big, dtype=torch.uint8, device="cuda")        # one workspace for every shape
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    for i in (0, 1, 2, 3, 4, 0, 2, 4, 1, 3, 3, 0):
        out, n, _ = ctx.match_pair(dev[i][0], dev[i][1], pc, ws=ws)
        assert ctx.pairs_host(out, n).tobytes() == ref[i], i
    # same buffers, same shape, new content: the cached tables still apply
    a2, b2 = _pair(SHAPES[0], 77)
    ref2 = _fresh(A, a2, b2)
    out = torch.zeros(200000, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    t1, t2 = dev[0][0].clone(), dev[0][1].clone()
    ctx.match_pair(t1, t2, pc, out, n_out, ws)
    first = ctx.pairs_host(out, n_out).tobytes()
    assert first == ref[0]
    t1.copy_(torch.from_numpy(a2))
    t2.copy_(torch.from_numpy(b2))
    ctx.match_pair(t1, t2, pc, out, n_out, ws)
    assert ctx.pairs_host(out, n_out).tobytes() == ref2
    # a workspace too small for a cached key is still refused
    with pytest.raises(A.AsiftError):
        ctx.match_pair(t1, t2, pc, out, n_out, ws[: 1024])
