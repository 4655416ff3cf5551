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
import ctypes as C

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


def _raw(A, L, fn, ctx, q, nq_cap, d_nq, t, nt_cap, d_nt):
    """One call through the C ABI with device-side counts d_nq / d_nt (int32
    tensors or None) and capacities nq_cap / nt_cap; returns the output bytes."""
    out = torch.zeros(max(nq_cap, 1) * 8, dtype=torch.uint8, device="cuda")
    acc = torch.zeros(max(nq_cap, 1), dtype=torch.uint8, device="cuda")
    nacc = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = lambda x: None if x is None else C.c_void_p(x.data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if fn == "noalloc":
        r = L.hamming_match_noalloc(p(q), nq_cap, p(d_nq), p(t), nt_cap, p(d_nt), 4, 5, p(out), p(acc), p(nacc), s)
    else:
        ws = torch.zeros(L.hamming_workspace_size(nq_cap, nt_cap), dtype=torch.uint8, device="cuda")
        r = L.hamming_match(ctx._ctx, p(q), nq_cap, p(d_nq), p(t), nt_cap, p(d_nt), 4, 5, p(out), p(acc), p(nacc),
                            p(ws), ws.numel(), s)
    assert r == A.ASIFT_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().tobytes(), acc.cpu().numpy().tobytes(), int(nacc.item())


def test_noalloc_device_counts_and_empty_train_set(A):
    """Counts read from the device (smaller than the capacities) and an empty
    train set, bit for bit against hamming_match on the same arguments."""
    L = A.load_library()
    ctx = A.Context()
    q, t = _pair(5_000, 4_000, 13)
    nq_d = torch.tensor([3_333], dtype=torch.int32, device="cuda")
    nt_d = torch.tensor([1_777], dtype=torch.int32, device="cuda")
    for d_nq, d_nt in ((nq_d, nt_d), (None, nt_d), (nq_d, None)):
        got = _raw(A, L, "noalloc", None, q, 5_000, d_nq, t, 4_000, d_nt)
        want = _raw(A, L, "ws", ctx, q, 5_000, d_nq, t, 4_000, d_nt)
        assert got == want and got[2] > 0
    zero = torch.zeros(1, dtype=torch.int32, device="cuda")
    for d_nt, nt_cap in ((zero, 4_000), (None, 0)):          # no train descriptors: no match, none accepted
        got = _raw(A, L, "noalloc", None, q, 5_000, None, t if nt_cap else None, nt_cap, d_nt)
        want = _raw(A, L, "ws", ctx, q, 5_000, None, t if nt_cap else None, nt_cap, d_nt)
        assert got == want and got[2] == 0
        m = np.frombuffer(got[0], dtype=A.MATCH_DTYPE)
        assert (m["best"] == -1).all() and (m["d1"] == 257).all()


def test_noalloc_rejects_sizes_beyond_its_limit(A):
    L = A.load_library()
    assert L.hamming_match_noalloc(None, 1_000_001, None, None, 0, None, 4, 5, None, None, None,
                                   None) == A.ASIFT_ERR_ARG
    assert L.hamming_match_noalloc(None, -1, None, None, 0, None, 4, 5, None, None, None, None) == A.ASIFT_ERR_ARG
