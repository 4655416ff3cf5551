"""The allocation-free matcher entry point, through the C ABI.

hamming_match_noalloc serves callers that may not allocate device memory (code
that a host framework hands only input and output buffers, and loops that
forbid cudaMalloc after start-up).  Its scratch is a fixed array inside the
library instead of a caller workspace.  Here it must give exactly the results
of the workspace-based hamming_match, on two calls in a row (the second call
smaller than the first, so stale scratch from the first would show), and it
must reject sizes beyond its stated limit.

This file is collected last on purpose, and it passes both on its own in a
fresh process and after the other tests.
"""
import numpy as np
import pytest
import torch

from paper_2503_03479_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    from paper_2503_03479_gb300 import build as B
    B.build()
    from paper_2503_03479_gb300 import asift
    assert torch.cuda.is_available()
    return asift


def _pair(nq, nt, seed):
    q = synth.random_descriptors(nq, seed)
    t = synth.random_descriptors(nt, seed + 1)
    t[5] = q[0]
    t[6] = q[0]                   # an exact tie
    t[9] = q[3] ^ 0x11            # a near-duplicate
    return torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda()


def test_noalloc_equals_workspace_matcher_on_two_calls(A):
    ctx = A.Context()
    # a large call (150k queries: the fixed array holds only 6 train slices of
    # partial keys for them, fewer than the workspace matcher uses), then a
    # smaller one
    for nq, nt, seed in ((150_000, 9_000, 11), (3_001, 2_049, 12)):
        q, t = _pair(nq, nt, seed)
        got = A.hamming_match_noalloc(q, t)
        want = ctx.hamming_match(q, t)
        for g, w in zip(got[:4], want[:4]):
            assert np.array_equal(g, w)
        assert got[4] == want[4]
        assert got[4] > 0


def test_noalloc_rejects_sizes_beyond_its_limit(A):
    L = A.load_library()
    assert L.hamming_match_noalloc(None, 1_000_001, None, None, 0, None, 4, 5, None, None, None,
                                   None) == A.ASIFT_ERR_ARG
    assert L.hamming_match_noalloc(None, -1, None, None, 0, None, 4, 5, None, None, None, None) == A.ASIFT_ERR_ARG
