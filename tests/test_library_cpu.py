"""Host-side checks of libasift that need no GPU: the library builds and loads,
exports every entry point of include/asift.h, rejects bad arguments, and its
host tables equal the oracle's (generated independently from the same
written definitions)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2503_03479_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def A():
    B.build()
    from paper_2503_03479_gb300 import asift
    asift.load_library()
    return asift


def _declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "asift.h")).read()
    return sorted(set(re.findall(r"^ASIFT_API\s+[\w\s\*]+?\b(\w+)\(", hdr, flags=re.M)))


def test_library_exports_every_declared_symbol(A):
    L = A.load_library()
    declared = _declared_symbols()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(A.EXPORTED) == declared
    # nothing but the C ABI is exported
    out = os.popen(f"nm -D --defined-only {A.LIB_PATH}").read()
    text = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert text == declared


@pytest.mark.parametrize("H,W,kmax", [(240, 320, 2), (768, 1024, 5), (3072, 4096, 6), (361, 487, 5), (1, 1, 3)])
def test_view_table_equals_oracle(A, H, W, kmax):
    a = A.view_table(H, W, kmax)
    b = O.view_table(H, W, kmax)
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert (x.k, x.j, x.W, x.H, x.Wr, x.Hr, x.Wv, x.Hv, x.K) == (y.k, y.j, y.W, y.H, y.Wr, y.Hr, y.Wv, y.Hv, y.K)
        assert (x.t, x.phi_deg, x.sigma, x.cq, x.sq, x.tq) == (y.t, y.phi_deg, y.sigma, y.cq, y.sq, y.tq)
        g = O.gauss_taps(y.sigma, y.K)
        assert np.array_equal(np.array(x.g[: y.K + 1], np.float32), g.astype(np.float32))


def test_make_view_equals_oracle(A):
    for t, phi in [(1.0, 90.0), (1.7, 33.3), (5.7, 179.0), (2.0, 0.0), (11.0, 45.0)]:
        x, y = A.make_view(123, 77, t, phi), O.make_view(123, 77, t, phi)
        assert (x.Wr, x.Hr, x.Wv, x.Hv, x.K, x.cq, x.sq, x.tq) == (y.Wr, y.Hr, y.Wv, y.Hv, y.K, y.cq, y.sq, y.tq)


def test_tables_equal_oracle(A):
    assert np.array_equal(A.pattern_table(), O.pattern())
    assert np.array_equal(A.pattern_table(12345), O.pattern(12345))
    assert np.array_equal(A.bin_table(), O.bin_table())
    for n0 in (15, 186, 1024, 4096):
        for l in range(10):
            assert A.level_size(n0, l) == O.level_size(n0, l)


def test_bad_arguments_are_rejected(A):
    L = A.load_library()
    n = C.c_int()
    assert L.asift_view_table(0, 10, 2, None, 0, C.byref(n)) == A.ASIFT_ERR_ARG
    assert L.asift_view_table(10, 10, 9, None, 0, C.byref(n)) == A.ASIFT_ERR_ARG
    assert L.asift_view_table(10, 10, 2, None, 0, None) == A.ASIFT_ERR_ARG
    v = A.ViewDesc()
    assert L.asift_make_view(10, 10, 0.5, 0.0, C.byref(v)) == A.ASIFT_ERR_ARG
    assert L.asift_pattern_table(1, None) == A.ASIFT_ERR_ARG
    assert L.match_pair_workspace_size(None, 10, 10, 10, 10, None) == 0
    assert L.hamming_match(None, None, 0, None, None, 0, None, 4, 5, None, None, None, None, 0, None) == A.ASIFT_ERR_ARG
    assert L.asift_read_status(None, 0, None, None) == A.ASIFT_ERR_ARG
    assert L.match_pair_view_counts(None, 10, 10, 10, 10, None, None, None, 0, None, None) == A.ASIFT_ERR_ARG
    assert L.asift_views_nearest(None, None, 10, 10, 10, None, 0, None, None, None, None, None, 0,
                                 None) == A.ASIFT_ERR_ARG
    for a in (3, 4, 2, 5):
        assert L.asift_views_lanczos(None, a, None, 10, 10, 10, None, 0, None, None, None, None, None, 0,
                                     None) == A.ASIFT_ERR_ARG
    assert L.asift_eval_pairs(None, None, None, 0, None, 3.0, None, 0, 9.0, None, None, None, None, None, 0,
                              None) == A.ASIFT_ERR_ARG
    assert L.asift_scale_coefficient(None, None, None, 0, None, None, 0, None) == A.ASIFT_ERR_ARG
    assert L.asift_plan_view_counts(None, 0, None, 0, None, None) == A.ASIFT_ERR_ARG
    assert L.asift_plan_eval(None, None, 3.0, None, 0, 9.0, None, 0, None) == A.ASIFT_ERR_ARG
    assert L.asift_plan_eval_outputs(None, None, 0, 0, None, None, None, None) == A.ASIFT_ERR_ARG
    assert L.asift_plan_eval_workspace_size(None, 16) == 0
    assert L.asift_sift(None, None, 100, 100, 100, 10, None, None, None, None, 0, None) == A.ASIFT_ERR_ARG
    assert L.asift_sift_workspace_size(8, 100, 10) == 0 and L.asift_sift_workspace_size(100, 100, 0) == 0
    assert 0 < L.asift_sift_workspace_size(240, 320, 100) < L.asift_sift_workspace_size(768, 1024, 100)


def test_context_without_gpu_fails_loudly(A):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = A.load_library()
    ctx = C.c_void_p()
    assert L.asift_ctx_create(C.byref(ctx), None, 1) == A.ASIFT_ERR_CUDA
    with pytest.raises(A.AsiftError):
        A.Context()


def test_workspace_sizes_are_monotone(A):
    L = A.load_library()
    assert L.hamming_workspace_size(1000, 2000) < L.hamming_workspace_size(40000, 40000)
    assert L.asift_views_workspace_size(240, 320, 10) < L.asift_views_workspace_size(768, 1024, 43)
    assert 0 < L.asift_eval_workspace_size(0, 0) <= L.asift_eval_workspace_size(1000, 64) \
        < L.asift_eval_workspace_size(43000, 1024)
    assert L.asift_eval_workspace_size(-1, 0) == 0 and L.asift_eval_workspace_size(10, -1) == 0
    assert L.asift_eval_workspace_size(1 << 27, 1) == 0 and L.asift_eval_workspace_size(10, (1 << 20) + 1) == 0
    assert 0 < L.asift_scale_coefficient_workspace_size(0) <= L.asift_scale_coefficient_workspace_size(43000)
    assert L.asift_scale_coefficient_workspace_size(-5) == 0


def test_view_sampling_matches_the_printed_rule(A):
    """The (t, phi) list of k <= 5 equals the table written out from the
    sampling rule printed in Sec. III-B (tests/golden), for the oracle and for
    the library alike."""
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "view_sampling_sec3b.json")))
    want = [(v["k"], v["j"], v["t"], v["phi_deg"]) for v in gold["views"]]
    assert len(want) == 43
    for tab in (O.view_table(768, 1024, 5), A.view_table(768, 1024, 5)):
        got = [(v.k, v.j, v.t, v.phi_deg) for v in tab]
        assert [(k, j) for k, j, _, _ in got] == [(k, j) for k, j, _, _ in want]
        for (_, _, t, phi), (_, _, tw, phiw) in zip(got, want):
            assert abs(t - tw) < 1e-12 and abs(phi - phiw) < 1e-9


@pytest.mark.parametrize("H,W,kmax,ds", [(768, 1024, 5, 0.5), (361, 487, 5, 0.5), (240, 320, 2, 1.25), (96, 128, 3, 0.0)])
def test_scaled_view_table_equals_oracle(A, H, W, kmax, ds):
    a = A.view_table(H, W, kmax, ds)
    b = O.view_table_scaled(H, W, kmax, ds)
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert (x.k, x.j, x.W, x.H, x.Wr, x.Hr, x.Wv, x.Hv, x.K) == (y.k, y.j, y.W, y.H, y.Wr, y.Hr, y.Wv, y.Hv, y.K)
        assert (x.t, x.phi_deg, x.sigma, x.s, x.cq, x.sq, x.tq) == (y.t, y.phi_deg, y.sigma, y.scale, y.cq, y.sq, y.tq)
    for t, phi, s in [(1.0, 0.0, 2.0), (3.3, 47.0, 1.75), (11.0, 90.0, 3.5)]:
        x, y = A.make_view(123, 77, t, phi, s), O.make_view(123, 77, t, phi, s)
        assert (x.Wr, x.Hr, x.Wv, x.Hv, x.K, x.cq, x.sq, x.tq, x.s) == (y.Wr, y.Hr, y.Wv, y.Hv, y.K, y.cq, y.sq, y.tq,
                                                                         y.scale)


def test_scaled_view_arguments_are_checked(A):
    L = A.load_library()
    n = C.c_int()
    assert L.asift_view_table_scaled(100, 100, 3, -0.5, None, 0, C.byref(n)) == A.ASIFT_ERR_ARG
    assert L.asift_view_table_scaled(100, 100, 3, 2.5, None, 0, C.byref(n)) == A.ASIFT_ERR_ARG
    v = A.ViewDesc()
    assert L.asift_make_view_scaled(100, 100, 2.0, 10.0, 0.5, C.byref(v)) == A.ASIFT_ERR_ARG
    assert L.asift_make_view_scaled(100, 100, 2.0, 10.0, 9.0, C.byref(v)) == A.ASIFT_ERR_ARG


def test_tuning_cache_round_trip(A, tmp_path):
    """The autotuner's choice persists per workload key; entries of another
    shape are ignored (searched again)."""
    path = str(tmp_path / "tuning.json")
    c = A.TuningCache(path)
    key = A.TuningCache.key([(768, 1024, 768, 1024), (480, 640, 360, 480)], 5, 8, 1000, "GB300")
    other = A.TuningCache.key([(768, 1024, 768, 1024)], 5, 8, 1000, "GB300", coarse=True)
    assert key != other and c.get(key) is None
    t = {"warp_grid": 456, "pyramid_grid": 0, "detect_grid": 912, "match_grid": 152, "match_target_items": 4,
         "match_engine": A.MATCH_TENSOR_CORES, "warp_seg": 512}
    c.put(key, t)
    assert A.TuningCache(path).get(key) == t and A.TuningCache(path).get(other) is None
    # the fields of the C struct, nothing else
    assert set(A.TuningCache.FIELDS) == set(A.Tuning().as_dict())
    with pytest.raises(ValueError):
        c.put(other, {"warp_grid": 1})
    import json
    raw = json.load(open(path))
    raw[other] = {"warp_grid": -1}
    json.dump(raw, open(path, "w"))
    assert A.TuningCache(path).get(other) is None
