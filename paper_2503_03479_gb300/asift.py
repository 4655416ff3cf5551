"""Thin ctypes binding of libasift (include/asift.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch provides device memory and the current CUDA stream.
Importing this module loads ``_build/libasift.so``; if it is missing the import
fails with an error telling how to build it (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libasift.so")

ASIFT_OK, ASIFT_ERR_ARG, ASIFT_ERR_CUDA, ASIFT_ERR_CAPACITY, ASIFT_ERR_TIMEOUT, ASIFT_ERR_NOMEM = 0, -1, -2, -3, -4, -5
_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_CAPACITY", -4: "ERR_TIMEOUT", -5: "ERR_NOMEM"}
MAX_GAUSS = 48
PATTERN_SEED = 250303479

EXPORTED = ["asift_ctx_create", "asift_ctx_destroy", "asift_ctx_orb_cfg", "asift_ctx_pattern", "asift_view_table",
            "asift_make_view", "asift_view_table_scaled", "asift_make_view_scaled", "asift_level_size", "asift_views_bytes", "asift_views_workspace_size", "asift_views", "asift_views_nearest", "asift_views_lanczos",
            "orb_workspace_size", "orb_extract", "hamming_workspace_size", "hamming_match",
            "match_pair_workspace_size", "match_pair", "match_pair_inspect", "match_pair_view_counts", "asift_sift_workspace_size", "asift_sift", "asift_scale_coefficient_workspace_size",
            "asift_scale_coefficient", "asift_eval_workspace_size",
            "asift_eval_pairs", "asift_read_status",
            "asift_launch_count", "asift_pattern_table", "asift_bin_table", "asift_profile_enable",
            "asift_profile_read", "hamming_match_noalloc", "asift_plan_create", "asift_plan_run",
            "asift_plan_pairs", "asift_plan_view_counts", "asift_plan_eval_workspace_size", "asift_plan_eval",
            "asift_plan_eval_outputs", "asift_plan_workspace", "asift_plan_set_tuning", "asift_plan_get_tuning",
            "asift_plan_autotune", "asift_plan_destroy", "asift_warp_shape_for", "asift_warp_workspace_size",
            "asift_warp_fwd", "asift_warp_bwd", "asift_ctx_set_match_engine", "asift_ctx_match_engine",
            "asift_ctx_set_test_hook", "asift_sift_match_workspace_size", "asift_sift_match", "asift_warp_loss",
            "asift_warp_adam"]
MATCH_AUTO, MATCH_CUDA_CORES, MATCH_TENSOR_CORES = 0, 1, 2
HOOK_CAND_CAP, HOOK_MATCH_STALL = 1, 2
INTERP_LANCZOS3, INTERP_NEAREST = 0, 1
PROF_STAGES = ["upload", "warp", "pyramid", "detect", "select", "orient_brief", "match", "pairs"]


class AsiftError(RuntimeError):
    def __init__(self, where: str, code: int):
        super().__init__(f"{where} failed: {_NAMES.get(code, code)}")
        self.code = code


class ViewDesc(C.Structure):
    _fields_ = [("k", C.c_int32), ("j", C.c_int32), ("W", C.c_int32), ("H", C.c_int32),
                ("Wr", C.c_int32), ("Hr", C.c_int32), ("Wv", C.c_int32), ("Hv", C.c_int32),
                ("K", C.c_int32), ("pad0", C.c_int32),
                ("t", C.c_double), ("phi_deg", C.c_double), ("sigma", C.c_double), ("s", C.c_double),
                ("cq", C.c_int64), ("sq", C.c_int64), ("tq", C.c_int64),
                ("g", C.c_float * MAX_GAUSS)]


class OrbCfg(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_features", C.c_int32), ("fast_threshold", C.c_int32),
                ("cand_per_mpx", C.c_int32)]


class PairCfg(C.Structure):
    _fields_ = [("kmax", C.c_int32), ("ratio_num", C.c_int32), ("ratio_den", C.c_int32), ("per_view", C.c_int32),
                ("coarse", C.c_int32), ("interp", C.c_int32), ("ds", C.c_double)]


class EvalResult(C.Structure):
    _fields_ = [("n_pairs", C.c_int32), ("n_unique", C.c_int32), ("r_num", C.c_int32), ("best_hyp", C.c_int32),
                ("n_inliers", C.c_int32), ("status", C.c_int32), ("ransac_th_sq", C.c_double),
                ("H", C.c_double * 9)]


class PairDesc(C.Structure):
    _fields_ = [("d_img1", C.c_void_p), ("H1", C.c_int32), ("W1", C.c_int32), ("pitch1", C.c_int32),
                ("d_img2", C.c_void_p), ("H2", C.c_int32), ("W2", C.c_int32), ("pitch2", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("warp_grid", C.c_int32), ("pyramid_grid", C.c_int32), ("detect_grid", C.c_int32),
                ("match_grid", C.c_int32), ("match_target_items", C.c_int32), ("match_engine", C.c_int32),
                ("warp_seg", C.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class WarpShape(C.Structure):
    _fields_ = [("Wr", C.c_int32), ("Hr", C.c_int32), ("Wv", C.c_int32), ("Hv", C.c_int32),
                ("K", C.c_int32), ("pad", C.c_int32)]


KP_DTYPE = np.dtype([("x", np.int16), ("y", np.int16), ("level", np.uint8), ("bin", np.uint8),
                     ("view", np.uint16), ("r25", np.int64)])
SIFT_KP_DTYPE = np.dtype([("x", np.float32), ("y", np.float32), ("sigma", np.float32), ("angle", np.float32),
                          ("response", np.float32), ("octave", np.int32), ("layer", np.int32), ("xo", np.float32),
                          ("yo", np.float32), ("so", np.float32), ("pad", np.int32, 2)])
MATCH_DTYPE = np.dtype([("best", np.int32), ("d1", np.uint16), ("d2", np.uint16)])
L2_MATCH_DTYPE = np.dtype([("best", np.int32), ("d1", np.float32), ("d2", np.float32)])
PAIR_DTYPE = np.dtype([("x1", np.float32), ("y1", np.float32), ("x2", np.float32), ("y2", np.float32),
                       ("q", np.int32), ("t", np.int32), ("d1", np.uint16), ("d2", np.uint16)])

_lib = None


def load_library():
    """Loads libasift.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libasift.so not found at {LIB_PATH}; build it with "
                          "`python -m paper_2503_03479_gb300.build` (needs nvcc)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, sz = C.c_void_p, C.c_int, C.c_int64, C.c_size_t
    P = C.POINTER
    sig = {
        "asift_ctx_create": (i32, [P(vp), P(OrbCfg), C.c_uint64]),
        "asift_ctx_destroy": (None, [vp]),
        "asift_ctx_orb_cfg": (i32, [vp, P(OrbCfg)]),
        "asift_ctx_set_match_engine": (i32, [vp, i32]),
        "asift_ctx_match_engine": (i32, [vp]),
        "asift_ctx_set_test_hook": (i32, [vp, i32, i64]),
        "asift_ctx_pattern": (i32, [vp, vp]),
        "asift_view_table": (i32, [i32, i32, i32, vp, i32, P(C.c_int)]),
        "asift_make_view": (i32, [i32, i32, C.c_double, C.c_double, P(ViewDesc)]),
        "asift_view_table_scaled": (i32, [i32, i32, i32, C.c_double, vp, i32, P(C.c_int)]),
        "asift_make_view_scaled": (i32, [i32, i32, C.c_double, C.c_double, C.c_double, P(ViewDesc)]),
        "asift_level_size": (i32, [i32, i32]),
        "asift_views_bytes": (i64, [vp, i32]),
        "asift_views_workspace_size": (sz, [i32, i32, i32]),
        "asift_views": (i32, [vp, vp, i32, i32, i32, vp, i32, vp, vp, vp, vp, vp, sz, vp]),
        "asift_views_nearest": (i32, [vp, vp, i32, i32, i32, vp, i32, vp, vp, vp, vp, vp, sz, vp]),
        "asift_views_lanczos": (i32, [vp, i32, vp, i32, i32, i32, vp, i32, vp, vp, vp, vp, vp, sz, vp]),
        "orb_workspace_size": (sz, [vp, vp, i32]),
        "orb_extract": (i32, [vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
        "hamming_workspace_size": (sz, [i32, i32]),
        "hamming_match": (i32, [vp, vp, i32, vp, vp, i32, vp, i32, i32, vp, vp, vp, vp, sz, vp]),
        "match_pair_workspace_size": (sz, [vp, i32, i32, i32, i32, P(PairCfg)]),
        "match_pair": (i32, [vp, vp, i32, i32, i32, vp, i32, i32, i32, P(PairCfg), vp, i32, vp, vp, sz, vp]),
        "match_pair_inspect": (i32, [vp, i32, i32, i32, i32, P(PairCfg), vp, vp, vp, vp, vp, vp, vp, vp]),
        "match_pair_view_counts": (i32, [vp, i32, i32, i32, i32, P(PairCfg), vp, vp, i32, vp, vp]),
        "asift_sift_workspace_size": (sz, [i32, i32, i32]),
        "asift_sift": (i32, [vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, sz, vp]),
        "asift_sift_match_workspace_size": (sz, [i32, i32]),
        "asift_sift_match": (i32, [vp, vp, i32, vp, vp, i32, vp, C.c_double, vp, vp, vp, vp, i32, vp, vp, sz, vp]),
        "asift_scale_coefficient_workspace_size": (sz, [i32]),
        "asift_scale_coefficient": (i32, [vp, vp, vp, i32, vp, vp, sz, vp]),
        "asift_eval_workspace_size": (sz, [i32, i32]),
        "asift_eval_pairs": (i32, [vp, vp, vp, i32, vp, C.c_double, vp, i32, C.c_double, vp, vp, vp, vp, vp, sz,
                                   vp]),
        "asift_read_status": (i32, [vp, i32, P(C.c_int32), vp]),
        "asift_launch_count": (i64, []),
        "asift_pattern_table": (i32, [C.c_uint64, vp]),
        "asift_bin_table": (i32, [vp]),
        "asift_profile_enable": (i32, [vp, i32]),
        "asift_profile_read": (i32, [vp, vp, i32]),
        "hamming_match_noalloc": (i32, [vp, i32, vp, vp, i32, vp, i32, i32, vp, vp, vp, vp]),
        "asift_plan_create": (i32, [vp, vp, i32, P(PairCfg), P(Tuning), i32, P(vp)]),
        "asift_plan_run": (i32, [vp, vp]),
        "asift_plan_pairs": (i32, [vp, i32, P(vp), P(C.c_int), P(vp)]),
        "asift_plan_view_counts": (i32, [vp, i32, vp, i32, vp, vp]),
        "asift_plan_eval_workspace_size": (sz, [vp, i32]),
        "asift_plan_eval": (i32, [vp, vp, C.c_double, vp, i32, C.c_double, vp, sz, vp]),
        "asift_plan_eval_outputs": (i32, [vp, vp, i32, i32, P(vp), P(vp), P(vp), P(vp)]),
        "asift_plan_workspace": (i32, [vp, P(vp), P(vp)]),
        "asift_plan_set_tuning": (i32, [vp, P(Tuning)]),
        "asift_plan_get_tuning": (i32, [vp, P(Tuning)]),
        "asift_plan_autotune": (i32, [vp, i32, P(Tuning)]),
        "asift_plan_destroy": (None, [vp]),
        "asift_warp_shape_for": (i32, [i32, i32, C.c_double, C.c_double, C.c_double, P(WarpShape)]),
        "asift_warp_workspace_size": (sz, [i32]),
        "asift_warp_fwd": (i32, [vp, vp, i32, i32, i32, vp, vp, C.c_double, vp, vp, vp, sz, vp]),
        "asift_warp_bwd": (i32, [vp, vp, i32, i32, i32, vp, vp, C.c_double, vp, vp, vp, vp, vp, sz, vp]),
        "asift_warp_loss": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
        "asift_warp_adam": (i32, [vp, i32, vp, vp, vp, vp, i32, vp, C.c_double, C.c_double, C.c_double, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(where: str, code: int):
    if code != ASIFT_OK:
        raise AsiftError(where, code)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def launch_count() -> int:
    return int(load_library().asift_launch_count())


def level_size(n0: int, l: int) -> int:
    return int(load_library().asift_level_size(n0, l))


def view_table(H: int, W: int, kmax: int, ds: float | None = None) -> list[ViewDesc]:
    """The views of the sampling rule (scale 1), or with ds the coarse stage's
    parameter groups (scale 1 + k ds)."""
    L = load_library()
    n = C.c_int()
    if ds is None:
        _check("asift_view_table", L.asift_view_table(H, W, kmax, None, 0, C.byref(n)))
        arr = (ViewDesc * n.value)()
        _check("asift_view_table", L.asift_view_table(H, W, kmax, arr, n.value, C.byref(n)))
    else:
        _check("asift_view_table_scaled", L.asift_view_table_scaled(H, W, kmax, float(ds), None, 0, C.byref(n)))
        arr = (ViewDesc * n.value)()
        _check("asift_view_table_scaled", L.asift_view_table_scaled(H, W, kmax, float(ds), arr, n.value, C.byref(n)))
    return list(arr)


def pattern_table(seed: int = PATTERN_SEED) -> np.ndarray:
    out = np.zeros((30, 256, 4), np.int8)
    _check("asift_pattern_table", load_library().asift_pattern_table(seed, out.ctypes.data_as(C.c_void_p)))
    return out


def bin_table() -> np.ndarray:
    out = np.zeros((30, 2), np.int64)
    _check("asift_bin_table", load_library().asift_bin_table(out.ctypes.data_as(C.c_void_p)))
    return out


def make_view(H: int, W: int, t: float, phi_deg: float, s: float = 1.0) -> ViewDesc:
    v = ViewDesc()
    _check("asift_make_view_scaled",
           load_library().asift_make_view_scaled(H, W, float(t), float(phi_deg), float(s), C.byref(v)))
    return v


def _view_array(views):
    arr = (ViewDesc * len(views))()
    for i, v in enumerate(views):
        arr[i] = v
    return arr


def view_offsets(views) -> np.ndarray:
    sizes = np.array([v.Wv * v.Hv for v in views], dtype=np.int64)
    return np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64), int(sizes.sum())


@dataclass
class ViewsOut:
    u8: torch.Tensor       # flat arena, view v at offsets[v], Hv x Wv
    mask: torch.Tensor
    f32: torch.Tensor | None
    offsets: np.ndarray
    views: list

    def view(self, i: int, which: str = "u8") -> torch.Tensor:
        v = self.views[i]
        buf = {"u8": self.u8, "mask": self.mask, "f32": self.f32}[which]
        o = int(self.offsets[i])
        return buf[o:o + v.Wv * v.Hv].view(v.Hv, v.Wv)


@dataclass
class OrbOut:
    kp: torch.Tensor        # (cap * 16) bytes of asift_keypoint
    desc: torch.Tensor      # (cap, 32) uint8
    view_count: torch.Tensor
    view_offset: torch.Tensor
    total: torch.Tensor     # int32 [1]

    def host(self):
        n = int(self.total.item())
        kp = self.kp[: n * 16].cpu().numpy().view(KP_DTYPE)
        return kp, self.desc[:n].cpu().numpy(), self.view_count.cpu().numpy(), self.view_offset.cpu().numpy()


def hamming_match_noalloc(q: torch.Tensor, t: torch.Tensor, num: int = 4, den: int = 5):
    """Matcher without a context or workspace (output buffers are the caller's).

    Returns (best, d1, d2, accepted, n_accepted) like Context.hamming_match."""
    L = load_library()
    nq, nt = q.shape[0], t.shape[0]
    dev = q.device
    out = torch.zeros(max(nq, 1) * 8, dtype=torch.uint8, device=dev)
    acc = torch.zeros(max(nq, 1), dtype=torch.uint8, device=dev)
    nacc = torch.zeros(1, dtype=torch.int32, device=dev)
    _check("hamming_match_noalloc", L.hamming_match_noalloc(_ptr(q) if nq else None, nq, None,
                                                            _ptr(t) if nt else None, nt, None, num, den,
                                                            _ptr(out), _ptr(acc), _ptr(nacc), _stream()))
    m = out[: nq * 8].cpu().numpy().view(MATCH_DTYPE)
    return (m["best"].copy(), m["d1"].astype(np.int32), m["d2"].astype(np.int32),
            acc[:nq].cpu().numpy().astype(bool), int(nacc.item()))


class Context:
    """A libasift context (pattern tables on the device) plus cached workspaces."""

    def __init__(self, n_levels: int = 4, n_features: int = 500, fast_threshold: int = 20,
                 cand_per_mpx: int = 60000, pattern_seed: int = PATTERN_SEED, device: int | None = None):
        self.L = load_library()
        if device is not None:
            torch.cuda.set_device(device)
        self.cfg = OrbCfg(n_levels, n_features, fast_threshold, cand_per_mpx)
        self._ctx = C.c_void_p()
        _check("asift_ctx_create", self.L.asift_ctx_create(C.byref(self._ctx), C.byref(self.cfg), pattern_seed))
        self._ws: dict = {}

    def close(self):
        if self._ctx:
            self.L.asift_ctx_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- workspace cache (allocation happens here, outside the library)
    def workspace(self, key, nbytes: int) -> torch.Tensor:
        w = self._ws.get(key)
        if w is None or w.numel() < nbytes:
            w = torch.zeros(max(nbytes, 256), dtype=torch.uint8, device="cuda")
            self._ws[key] = w
        return w

    # -- matcher engine (same results; speed only)
    def set_match_engine(self, engine: int):
        """MATCH_AUTO, MATCH_CUDA_CORES or MATCH_TENSOR_CORES for hamming_match and match_pair."""
        _check("asift_ctx_set_match_engine", self.L.asift_ctx_set_match_engine(self._ctx, int(engine)))

    def set_test_hook(self, hook: int, value: int):
        """Failure-path test hooks (HOOK_CAND_CAP, HOOK_MATCH_STALL; 0 turns one off)."""
        _check("asift_ctx_set_test_hook", self.L.asift_ctx_set_test_hook(self._ctx, int(hook), int(value)))

    @property
    def match_engine(self) -> int:
        """The engine a call would use now (MATCH_CUDA_CORES or MATCH_TENSOR_CORES)."""
        return int(self.L.asift_ctx_match_engine(self._ctx))

    def profile(self, on: bool = True):
        _check("asift_profile_enable", self.L.asift_profile_enable(self._ctx, int(on)))

    def profile_read(self) -> dict:
        ms = np.zeros(len(PROF_STAGES), np.float32)
        _check("asift_profile_read", self.L.asift_profile_read(self._ctx, ms.ctypes.data_as(C.c_void_p), len(ms)))
        return dict(zip(PROF_STAGES, ms.tolist()))

    def pattern(self) -> np.ndarray:
        out = np.zeros((30, 256, 4), np.int8)
        _check("asift_ctx_pattern", self.L.asift_ctx_pattern(self._ctx, out.ctypes.data_as(C.c_void_p)))
        return out

    def read_status(self, ws: torch.Tensor, clear: bool = True) -> int:
        st = C.c_int32()
        _check("asift_read_status", self.L.asift_read_status(_ptr(ws), int(clear), C.byref(st), _stream()))
        return st.value

    # -- asift_views
    def views(self, img: torch.Tensor, views, with_f32: bool = False, nearest: bool = False,
              lanczos: int | None = None) -> ViewsOut:
        """The views of one uint8 image: Lanczos-3 (default), nearest=True for the coarse stage's
        nearest-neighbour views, lanczos=a (3 or 4) for the precise stage's Lanczos-a kernel."""
        assert img.is_cuda and img.dtype == torch.uint8 and img.dim() == 2
        H, W = img.shape
        pitch = img.stride(0)
        offs, total = view_offsets(views)
        u8 = torch.empty(max(total, 1), dtype=torch.uint8, device=img.device)
        mask = torch.empty_like(u8)
        f32 = torch.empty(max(total, 1), dtype=torch.float32, device=img.device) if with_f32 else None
        nbytes = self.L.asift_views_workspace_size(H, W, len(views))
        ws = self.workspace("views", nbytes)
        arr = _view_array(views)
        rest = (_ptr(img), H, W, pitch, arr, len(views), offs.ctypes.data_as(C.c_void_p), _ptr(f32), _ptr(u8),
                _ptr(mask), _ptr(ws), ws.numel(), _stream())
        if lanczos is not None:
            _check("asift_views_lanczos", self.L.asift_views_lanczos(self._ctx, int(lanczos), *rest))
        else:
            fn = "asift_views_nearest" if nearest else "asift_views"
            _check(fn, getattr(self.L, fn)(self._ctx, *rest))
        return ViewsOut(u8, mask, f32, offs, list(views))

    # -- orb_extract
    def orb_extract(self, vo: ViewsOut) -> OrbOut:
        views = vo.views
        nv = len(views)
        cap = nv * self.cfg.n_features
        arr = _view_array(views)
        nbytes = self.L.orb_workspace_size(self._ctx, arr, nv)
        ws = self.workspace("orb", nbytes)
        dev = vo.u8.device
        kp = torch.zeros(cap * 16, dtype=torch.uint8, device=dev)
        desc = torch.zeros((cap, 32), dtype=torch.uint8, device=dev)
        vc = torch.zeros(nv, dtype=torch.int32, device=dev)
        vof = torch.zeros(nv, dtype=torch.int32, device=dev)
        total = torch.zeros(1, dtype=torch.int32, device=dev)
        _check("orb_extract", self.L.orb_extract(self._ctx, _ptr(vo.u8), _ptr(vo.mask), arr, nv,
                                                 vo.offsets.ctypes.data_as(C.c_void_p), _ptr(kp), _ptr(desc),
                                                 _ptr(vc), _ptr(vof), _ptr(total), _ptr(ws), ws.numel(), _stream()))
        self.last_orb_ws = ws
        return OrbOut(kp, desc, vc, vof, total)

    # -- hamming_match
    def hamming_match(self, q: torch.Tensor, t: torch.Tensor, num: int = 4, den: int = 5):
        """q: (nq, 32) uint8, t: (nt, 32) uint8 on the GPU -> (best, d1, d2, accepted, n_accepted)."""
        nq, nt = q.shape[0], t.shape[0]
        dev = q.device
        out = torch.zeros(max(nq, 1) * 8, dtype=torch.uint8, device=dev)
        acc = torch.zeros(max(nq, 1), dtype=torch.uint8, device=dev)
        nacc = torch.zeros(1, dtype=torch.int32, device=dev)
        ws = self.workspace("hamming", self.L.hamming_workspace_size(nq, nt))
        _check("hamming_match", self.L.hamming_match(self._ctx, _ptr(q) if nq else None, nq, None,
                                                     _ptr(t) if nt else None, nt, None, num, den, _ptr(out),
                                                     _ptr(acc), _ptr(nacc), _ptr(ws), ws.numel(), _stream()))
        m = out[: nq * 8].cpu().numpy().view(MATCH_DTYPE)
        return (m["best"].copy(), m["d1"].astype(np.int32), m["d2"].astype(np.int32),
                acc[:nq].cpu().numpy().astype(bool), int(nacc.item()))

    # -- hamming_match_noalloc (no workspace: the library's fixed scratch array)
    def hamming_match_noalloc(self, q: torch.Tensor, t: torch.Tensor, num: int = 4, den: int = 5):
        """As hamming_match, through the allocation-free entry point."""
        return hamming_match_noalloc(q, t, num, den)

    # -- match_pair
    def pair_cfg(self, kmax: int = 5, num: int = 4, den: int = 5, per_view: bool = False, coarse: bool = False,
                 ds: float = 0.5, nearest: bool = False) -> PairCfg:
        """coarse=True: image 1 takes the (t, phi, s) parameter groups with s = 1 + k ds, image 2 the
        identity view only (the coarse stage of Sec. 3); nearest=True: nearest-neighbour views."""
        return PairCfg(kmax, num, den, int(per_view), int(coarse), INTERP_NEAREST if nearest else INTERP_LANCZOS3,
                       float(ds))

    @staticmethod
    def pair_views(shape, pc: PairCfg, image: int) -> list:
        """View table of image 0 or 1 of a pair under pc."""
        H, W = shape
        if not pc.coarse:
            return view_table(H, W, pc.kmax)
        return view_table(H, W, 0) if image else view_table(H, W, pc.kmax, pc.ds)

    def match_pair_workspace(self, shape1, shape2, pc: PairCfg) -> torch.Tensor:
        n = self.L.match_pair_workspace_size(self._ctx, shape1[0], shape1[1], shape2[0], shape2[1], C.byref(pc))
        if n == 0:
            raise AsiftError("match_pair_workspace_size", ASIFT_ERR_ARG)
        return self.workspace(("pair", tuple(shape1), tuple(shape2), pc.kmax, pc.per_view, pc.coarse, pc.ds,
                               pc.interp), n)

    def match_pair(self, img1: torch.Tensor, img2: torch.Tensor, pc: PairCfg, out: torch.Tensor | None = None,
                   n_out: torch.Tensor | None = None, ws: torch.Tensor | None = None):
        """Whole hot path for one pair.  Returns (pairs byte buffer, count tensor, workspace)."""
        H1, W1 = img1.shape
        H2, W2 = img2.shape
        if ws is None:
            ws = self.match_pair_workspace((H1, W1), (H2, W2), pc)
        n1 = len(self.pair_views((H1, W1), pc, 0))
        cap = n1 * self.cfg.n_features
        if out is None:
            out = torch.zeros(max(cap, 1) * PAIR_DTYPE.itemsize, dtype=torch.uint8, device=img1.device)
        if n_out is None:
            n_out = torch.zeros(1, dtype=torch.int32, device=img1.device)
        cap = out.numel() // PAIR_DTYPE.itemsize
        _check("match_pair", self.L.match_pair(self._ctx, _ptr(img1), H1, W1, img1.stride(0), _ptr(img2), H2, W2,
                                               img2.stride(0), C.byref(pc), _ptr(out), cap, _ptr(n_out), _ptr(ws),
                                               ws.numel(), _stream()))
        return out, n_out, ws

    def pairs_host(self, out: torch.Tensor, n_out: torch.Tensor) -> np.ndarray:
        n = int(n_out.item())
        cap = out.numel() // PAIR_DTYPE.itemsize
        return out[: min(n, cap) * PAIR_DTYPE.itemsize].cpu().numpy().view(PAIR_DTYPE)

    def eval_pairs(self, out: torch.Tensor, n_out: torch.Tensor, H_true=None, th_sq: float = 3.0,
                   rnd: torch.Tensor | None = None, ransac_th_sq: float = 9.0, counts: bool = False):
        """Duplicate removal, Eq. (5)-(6) precision count against H_true (3x3, image 1 -> 2), RANSAC
        over rnd (device int32 (n_hyp, 4), read as uint32) and the Eq. (7) inliers, on match_pair's
        output.  Returns (unique pairs, inlier mask, per-hypothesis counts or None, result bytes);
        read the result with eval_result()."""
        cap = out.numel() // PAIR_DTYPE.itemsize
        n_hyp = 0 if rnd is None else rnd.shape[0]
        nbytes = self.L.asift_eval_workspace_size(cap, n_hyp)
        if nbytes == 0:
            raise AsiftError("asift_eval_workspace_size", ASIFT_ERR_ARG)
        ws = self.workspace(("eval", cap, n_hyp), nbytes)
        dev = out.device
        unique = torch.empty(max(cap, 1) * PAIR_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        inl = torch.empty(max(cap, 1), dtype=torch.uint8, device=dev)
        cnt = torch.empty(max(n_hyp, 1), dtype=torch.int32, device=dev) if counts else None
        res = torch.empty(C.sizeof(EvalResult), dtype=torch.uint8, device=dev)
        Hh = None
        if H_true is not None:
            Hh = (C.c_double * 9)(*[float(x) for x in np.asarray(H_true, dtype=np.float64).reshape(9)])
        _check("asift_eval_pairs",
               self.L.asift_eval_pairs(self._ctx, _ptr(out), _ptr(n_out), cap, Hh, float(th_sq),
                                       _ptr(rnd) if rnd is not None else None, n_hyp, float(ransac_th_sq),
                                       _ptr(unique), _ptr(inl), _ptr(cnt) if cnt is not None else None, _ptr(res),
                                       _ptr(ws), ws.numel(), _stream()))
        return unique, inl, cnt, res

    def sift_raw(self, img: torch.Tensor, max_kp: int = 20000):
        """asift_sift on a uint8 CUDA image: device (keypoints, descriptors, count) in append order."""
        assert img.is_cuda and img.dtype == torch.uint8 and img.dim() == 2
        H, W = img.shape
        nbytes = self.L.asift_sift_workspace_size(H, W, max_kp)
        if nbytes == 0:
            raise AsiftError("asift_sift_workspace_size", ASIFT_ERR_ARG)
        ws = self.workspace(("sift", H, W, max_kp), nbytes)
        kp = torch.empty(max_kp * SIFT_KP_DTYPE.itemsize, dtype=torch.uint8, device=img.device)
        desc = torch.empty((max_kp, 128), dtype=torch.float32, device=img.device)
        n = torch.zeros(1, dtype=torch.int32, device=img.device)
        _check("asift_sift", self.L.asift_sift(self._ctx, _ptr(img), H, W, img.stride(0), max_kp, _ptr(kp),
                                               _ptr(desc), _ptr(n), _ptr(ws), ws.numel(), _stream()))
        return kp, desc, n

    def sift(self, img: torch.Tensor, max_kp: int = 20000):
        """SIFT keypoints (SIFT_KP_DTYPE) and descriptors (float32, n x 128), host copies sorted by
        response (descending), then y, x, angle."""
        kp, desc, n = self.sift_raw(img, max_kp)
        k = min(int(n.item()), max_kp)
        kps = kp[: k * SIFT_KP_DTYPE.itemsize].cpu().numpy().view(SIFT_KP_DTYPE)
        d = desc[:k].cpu().numpy()
        order = np.lexsort((kps["angle"], kps["x"], kps["y"], -kps["response"]))
        return kps[order], d[order]

    def sift_match(self, dq: torch.Tensor, dt: torch.Tensor, ratio: float = 0.8, n_q: torch.Tensor | None = None,
                   n_t: torch.Tensor | None = None, kq: torch.Tensor | None = None, kt: torch.Tensor | None = None,
                   cap: int | None = None):
        """L2 SIFT matching (asift_sift_match): dq (nq, 128) and dt (nt, 128) fp32 CUDA
        descriptors, optional device counts n_q / n_t (int32 [1]) and keypoint buffers kq / kt
        (asift_sift_kp bytes, as sift_raw returns them).  Returns the device per-query results
        (L2_MATCH_DTYPE bytes), and with keypoints the accepted pairs (PAIR_DTYPE bytes) and
        their count."""
        nq, nt = dq.shape[0], dt.shape[0]
        dev = dq.device
        ws = self.workspace(("sift_match", nq, nt), self.L.asift_sift_match_workspace_size(nq, nt))
        out = torch.empty(max(nq, 1) * L2_MATCH_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        pairs = n_pairs = None
        if kq is not None and kt is not None:
            cap = nq if cap is None else cap
            pairs = torch.empty(max(cap, 1) * PAIR_DTYPE.itemsize, dtype=torch.uint8, device=dev)
            n_pairs = torch.zeros(1, dtype=torch.int32, device=dev)
        _check("asift_sift_match",
               self.L.asift_sift_match(self._ctx, _ptr(dq) if nq else None, nq, _ptr(n_q), _ptr(dt) if nt else None,
                                       nt, _ptr(n_t), float(ratio), _ptr(kq), _ptr(kt), _ptr(out), _ptr(pairs),
                                       cap or 0, _ptr(n_pairs), _ptr(ws), ws.numel(), _stream()))
        self.last_sift_match_ws = ws
        return out, pairs, n_pairs

    def scale_coefficient(self, out: torch.Tensor, n_out: torch.Tensor) -> torch.Tensor:
        """Eq. (1) over match_pair's output: a device float64 tensor of one element."""
        cap = out.numel() // PAIR_DTYPE.itemsize
        ws = self.workspace(("scale", cap), self.L.asift_scale_coefficient_workspace_size(cap))
        f = torch.empty(1, dtype=torch.float64, device=out.device)
        _check("asift_scale_coefficient", self.L.asift_scale_coefficient(self._ctx, _ptr(out), _ptr(n_out), cap,
                                                                         _ptr(f), _ptr(ws), ws.numel(), _stream()))
        return f

    def base_image(self, img1: torch.Tensor, img2: torch.Tensor, pc: PairCfg):
        """Sec. III-A: f1 on image 1 -> 2's accepted pairs, f2 on image 2 -> 1's; the reference is
        image 0 when f1 > f2, else image 1.  Returns (f1, f2, reference index)."""
        f = []
        for a, b in ((img1, img2), (img2, img1)):
            out, n, _ = self.match_pair(a, b, pc)
            f.append(float(self.scale_coefficient(out, n).item()))
        return f[0], f[1], 0 if f[0] > f[1] else 1

    @staticmethod
    def eval_result(res: torch.Tensor) -> EvalResult:
        b = res.cpu().numpy().tobytes()
        return EvalResult.from_buffer_copy(b)

    def view_counts(self, shape1, shape2, pc: PairCfg, ws: torch.Tensor):
        """Accepted matches per image-1 view of the last match_pair on ws, and the
        view with the most (lowest index on ties): device int32 tensors."""
        n1 = len(self.pair_views(shape1, pc, 0))
        counts = torch.empty(n1, dtype=torch.int32, device=ws.device)
        best = torch.empty(1, dtype=torch.int32, device=ws.device)
        _check("match_pair_view_counts",
               self.L.match_pair_view_counts(self._ctx, shape1[0], shape1[1], shape2[0], shape2[1], C.byref(pc),
                                             _ptr(ws), _ptr(counts), n1, _ptr(best), _stream()))
        return counts, best

    def inspect_pair(self, shape1, shape2, pc: PairCfg, ws: torch.Tensor):
        """Pooled keypoints / descriptors / matches of the last match_pair on ws (host copies)."""
        ptrs = [C.c_void_p() for _ in range(7)]
        _check("match_pair_inspect", self.L.match_pair_inspect(self._ctx, shape1[0], shape1[1], shape2[0], shape2[1],
                                                               C.byref(pc), _ptr(ws), *[C.byref(p) for p in ptrs]))
        torch.cuda.synchronize()
        base = ws.data_ptr()

        def sl(p, nbytes):
            o = p.value - base
            return ws[o:o + nbytes].cpu().numpy()

        n1 = int(sl(ptrs[2], 4).view(np.int32)[0])
        n2 = int(sl(ptrs[5], 4).view(np.int32)[0])
        kp1 = sl(ptrs[0], n1 * 16).view(KP_DTYPE)
        d1 = sl(ptrs[1], n1 * 32).reshape(n1, 32)
        kp2 = sl(ptrs[3], n2 * 16).view(KP_DTYPE)
        d2 = sl(ptrs[4], n2 * 32).reshape(n2, 32)
        m = sl(ptrs[6], n1 * 8).view(MATCH_DTYPE)
        return kp1, d1, kp2, d2, m


class TuningCache:
    """Autotuner results kept across runs in a JSON file: one launch-shape choice
    (Plan.tuning()) per workload key, so that a later plan over the same
    workload skips the search (Plan(..., tuning=cache.get(key)))."""

    FIELDS = ("warp_grid", "pyramid_grid", "detect_grid", "match_grid", "match_target_items", "match_engine",
              "warp_seg")

    def __init__(self, path: str):
        self.path = path
        self._d: dict = {}
        if os.path.exists(path):
            import json
            with open(path) as f:
                self._d = json.load(f)

    @staticmethod
    def key(shapes, kmax: int, n_levels: int, n_features: int, device: str, coarse: bool = False,
            nearest: bool = False) -> str:
        """The workload: every pair's (H1, W1, H2, W2), the view and ORB configuration and the device."""
        dims = ";".join(",".join(str(int(v)) for v in s) for s in shapes)
        return f"{device}|k{kmax}|L{n_levels}|N{n_features}|c{int(coarse)}|n{int(nearest)}|{dims}"

    def get(self, key: str):
        t = self._d.get(key)
        if t is None:
            return None
        if set(t) != set(self.FIELDS) or not all(isinstance(v, int) and v >= 0 for v in t.values()):
            return None                      # written by another version: search again
        return dict(t)

    def put(self, key: str, tuning: dict):
        if set(tuning) != set(self.FIELDS):
            raise ValueError("not a plan tuning")
        self._d[key] = {k: int(tuning[k]) for k in self.FIELDS}
        import json
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self._d, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


class Plan:
    """Batched form: all views of many pairs, one launch per stage, replayed
    from a CUDA graph.  The images (uint8 CUDA tensors) are captured by
    address: update them in place between runs."""

    def __init__(self, ctx: Context, imgs1, imgs2, kmax: int = 5, num: int = 4, den: int = 5,
                 tuning: dict | None = None, use_graph: bool = True, coarse: bool = False, ds: float = 0.5,
                 nearest: bool = False):
        self.ctx = ctx
        self.L = ctx.L
        self.imgs = list(zip(imgs1, imgs2))      # keep the tensors alive
        arr = (PairDesc * len(self.imgs))()
        for i, (a, b) in enumerate(self.imgs):
            assert a.is_cuda and a.dtype == torch.uint8 and b.is_cuda and b.dtype == torch.uint8
            arr[i] = PairDesc(a.data_ptr(), a.shape[0], a.shape[1], a.stride(0),
                              b.data_ptr(), b.shape[0], b.shape[1], b.stride(0))
        pc = PairCfg(kmax, num, den, 0, int(coarse), INTERP_NEAREST if nearest else INTERP_LANCZOS3, float(ds))
        self.pc = pc
        tn = Tuning(**tuning) if tuning else None
        self._p = C.c_void_p()
        torch.cuda.synchronize()
        _check("asift_plan_create", self.L.asift_plan_create(ctx._ctx, arr, len(self.imgs), C.byref(pc),
                                                             C.byref(tn) if tn else None, int(use_graph),
                                                             C.byref(self._p)))

    def close(self):
        if self._p:
            self.L.asift_plan_destroy(self._p)
            self._p = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self):
        _check("asift_plan_run", self.L.asift_plan_run(self._p, _stream()))

    def tuning(self) -> dict:
        t = Tuning()
        _check("asift_plan_get_tuning", self.L.asift_plan_get_tuning(self._p, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, tuning: dict):
        t = Tuning(**tuning)
        _check("asift_plan_set_tuning", self.L.asift_plan_set_tuning(self._p, C.byref(t)))

    def autotune(self, reps: int = 3) -> dict:
        t = Tuning()
        _check("asift_plan_autotune", self.L.asift_plan_autotune(self._p, reps, C.byref(t)))
        return t.as_dict()

    def workspace(self):
        ws, cnt = C.c_void_p(), C.c_void_p()
        _check("asift_plan_workspace", self.L.asift_plan_workspace(self._p, C.byref(ws), C.byref(cnt)))
        return ws.value, cnt.value

    def status(self) -> int:
        ws, _ = self.workspace()
        st = C.c_int32()
        _check("asift_read_status", self.L.asift_read_status(C.c_void_p(ws), 1, C.byref(st), _stream()))
        return st.value

    def pool_counts(self) -> np.ndarray:
        _, cnt = self.workspace()
        return device_view(cnt, (2 * len(self.imgs),), "<i4").cpu().numpy()

    def view_counts(self, i: int):
        """Accepted matches per image-1 view of pair i and the view with the most (device int32)."""
        a, _ = self.imgs[i]
        n1 = len(Context.pair_views(tuple(a.shape), self.pc, 0))
        counts = torch.empty(n1, dtype=torch.int32, device=a.device)
        best = torch.empty(1, dtype=torch.int32, device=a.device)
        _check("asift_plan_view_counts",
               self.L.asift_plan_view_counts(self._p, i, _ptr(counts), n1, _ptr(best), _stream()))
        return counts, best

    def evaluate(self, H_true=None, th_sq: float = 3.0, rnd: torch.Tensor | None = None,
                 ransac_th_sq: float = 9.0, read: bool = True):
        """asift_eval_pairs on every pair of the last run, one launch per stage.  H_true: a list
        of 3x3 homographies (one per pair) or None; rnd: device int32 (n_hyp, 4), read as uint32.
        Returns the per-pair EvalResult list; eval_outputs(i) gives pair i's device outputs."""
        n_hyp = 0 if rnd is None else rnd.shape[0]
        nbytes = self.L.asift_plan_eval_workspace_size(self._p, n_hyp)
        if nbytes == 0:
            raise AsiftError("asift_plan_eval_workspace_size", ASIFT_ERR_ARG)
        if getattr(self, "_eval_ws", None) is None or self._eval_ws.numel() < nbytes:
            self._eval_ws = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
        self._eval_hyp = n_hyp
        Hh = None
        if H_true is not None:
            flat = np.concatenate([np.asarray(h, dtype=np.float64).reshape(9) for h in H_true])
            Hh = (C.c_double * len(flat))(*flat.tolist())
        _check("asift_plan_eval", self.L.asift_plan_eval(self._p, Hh, float(th_sq), _ptr(rnd), n_hyp,
                                                         float(ransac_th_sq), _ptr(self._eval_ws),
                                                         self._eval_ws.numel(), _stream()))
        if not read:
            return None
        torch.cuda.synchronize()
        return [self._eval_result(i) for i in range(len(self.imgs))]

    def _eval_outputs(self, i: int):
        ptrs = [C.c_void_p() for _ in range(4)]
        _check("asift_plan_eval_outputs",
               self.L.asift_plan_eval_outputs(self._p, _ptr(self._eval_ws), self._eval_hyp, i,
                                              *[C.byref(q) for q in ptrs]))
        return [q.value for q in ptrs]

    def _eval_result(self, i: int) -> EvalResult:
        base = self._eval_ws.data_ptr()
        o = self._eval_outputs(i)[3] - base
        return EvalResult.from_buffer_copy(self._eval_ws[o:o + C.sizeof(EvalResult)].cpu().numpy().tobytes())

    def eval_outputs(self, i: int, n_unique: int):
        """Pair i's kept pairs (PAIR_DTYPE), inlier mask and per-hypothesis counts (host copies)."""
        base = self._eval_ws.data_ptr()
        u, m, c, _ = self._eval_outputs(i)
        uq = self._eval_ws[u - base:u - base + n_unique * PAIR_DTYPE.itemsize].cpu().numpy().view(PAIR_DTYPE)
        inl = self._eval_ws[m - base:m - base + n_unique].cpu().numpy().astype(bool)
        cnt = self._eval_ws[c - base:c - base + 4 * self._eval_hyp].cpu().numpy().view(np.int32)
        return uq, inl, cnt

    def pairs(self, i: int) -> np.ndarray:
        ptr, cap, dn = C.c_void_p(), C.c_int(), C.c_void_p()
        _check("asift_plan_pairs", self.L.asift_plan_pairs(self._p, i, C.byref(ptr), C.byref(cap), C.byref(dn)))
        k = min(int(device_view(dn.value, (1,), "<i4").item()), cap.value)
        if k == 0:
            return np.zeros(0, PAIR_DTYPE)
        return device_view(ptr.value, (k * PAIR_DTYPE.itemsize,), "|u1").cpu().numpy().view(PAIR_DTYPE)


class _DevPtr:
    """A raw device pointer exposed through __cuda_array_interface__ so that
    torch can view the library's own buffers without copying."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr: int, shape, typestr: str) -> torch.Tensor:
    torch.cuda.synchronize()
    return torch.as_tensor(_DevPtr(ptr, shape, typestr), device="cuda")


# ---------------------------------------------------------------- differentiable warp
@dataclass
class WarpLayout:
    """Fixed sizes of n differentiable views (from their initial parameters)."""
    shapes: object          # ctypes array of WarpShape
    voff: np.ndarray        # int64 element offsets of each view in the flat output
    total: int
    t_max: float
    H: int
    W: int

    def view(self, flat: torch.Tensor, i: int) -> torch.Tensor:
        s = self.shapes[i]
        o = int(self.voff[i])
        return flat[o:o + s.Wv * s.Hv].view(s.Hv, s.Wv)


def warp_layout(H: int, W: int, t0, phi0, t_max: float) -> WarpLayout:
    n = len(t0)
    arr = (WarpShape * n)()
    L = load_library()
    for i in range(n):
        _check("asift_warp_shape_for", L.asift_warp_shape_for(H, W, float(t0[i]), float(phi0[i]), float(t_max),
                                                              C.byref(arr[i])))
    sizes = np.array([arr[i].Wv * arr[i].Hv for i in range(n)], np.int64)
    voff = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return WarpLayout(arr, voff, int(sizes.sum()), float(t_max), H, W)


def warp_forward(ctx: Context, u: torch.Tensor, params: torch.Tensor, lay: WarpLayout) -> torch.Tensor:
    """u: (n, H, W) fp32 CUDA; params: (n, 4) fp64 CUDA (t, phi deg, tx, ty) -> flat views."""
    n = u.shape[0]
    u = u.contiguous()
    params = params.contiguous()
    out = torch.empty(max(lay.total, 1), dtype=torch.float32, device=u.device)
    ws = ctx.workspace("warp", ctx.L.asift_warp_workspace_size(n))
    _check("asift_warp_fwd", ctx.L.asift_warp_fwd(ctx._ctx, _ptr(u), lay.H, lay.W, n, _ptr(params), lay.shapes,
                                                  lay.t_max, _ptr(out), lay.voff.ctypes.data_as(C.c_void_p),
                                                  _ptr(ws), ws.numel(), _stream()))
    return out


def warp_backward(ctx: Context, u: torch.Tensor, params: torch.Tensor, lay: WarpLayout, vbar: torch.Tensor,
                  image_grad: bool = True):
    """(image gradient or None, parameter gradients (n, 4) fp64)."""
    n = u.shape[0]
    u = u.contiguous()
    params = params.contiguous()
    vbar = vbar.contiguous().to(torch.float32)
    ubar = torch.empty_like(u) if image_grad else None
    pbar = torch.empty((n, 4), dtype=torch.float64, device=u.device)
    ws = ctx.workspace("warp_bwd", ctx.L.asift_warp_workspace_size(n))
    _check("asift_warp_bwd", ctx.L.asift_warp_bwd(ctx._ctx, _ptr(u), lay.H, lay.W, n, _ptr(params), lay.shapes,
                                                  lay.t_max, _ptr(vbar), lay.voff.ctypes.data_as(C.c_void_p),
                                                  _ptr(ubar), _ptr(pbar), _ptr(ws), ws.numel(), _stream()))
    return ubar, pbar


class WarpFunction(torch.autograd.Function):
    """Differentiable Gaussian + Lanczos-3 view warp; the backward is the
    library's hand-written adjoint (canvas and blur recomputed)."""

    @staticmethod
    def forward(fctx, u, params, ctx: Context, lay: WarpLayout):
        fctx.save_for_backward(u, params)
        fctx.lib_ctx = ctx
        fctx.lay = lay
        return warp_forward(ctx, u, params, lay)

    @staticmethod
    def backward(fctx, vbar):
        u, params = fctx.saved_tensors
        ubar, pbar = warp_backward(fctx.lib_ctx, u, params, fctx.lay, vbar)
        return (ubar if fctx.needs_input_grad[0] else None,
                pbar if fctx.needs_input_grad[1] else None, None, None)


def warp_loss(ctx: Context, v: torch.Tensor, target: torch.Tensor, lay: WarpLayout, with_grad: bool = True):
    """Per-view mean squared photometric error (fp64 (n,)) and its gradient (flat fp32 or None)."""
    n = len(lay.voff)
    loss = torch.empty(n, dtype=torch.float64, device=v.device)
    vbar = torch.empty_like(v) if with_grad else None
    ws = ctx.workspace("warp_loss", ctx.L.asift_warp_workspace_size(n))
    _check("asift_warp_loss", ctx.L.asift_warp_loss(ctx._ctx, n, lay.shapes, lay.voff.ctypes.data_as(C.c_void_p),
                                                    _ptr(v), _ptr(target), _ptr(loss), _ptr(vbar), _ptr(ws),
                                                    ws.numel(), _stream()))
    return loss, vbar


def refine(ctx: Context, u: torch.Tensor, target: torch.Tensor, lay: WarpLayout, theta0: torch.Tensor,
           steps: int = 20, lr=(0.1, 2.0, 1.0, 1.0), decay: float = 0.88, t_range=(1.0, None)):
    """Photometric descent of the view parameters: Adam (step sizes lr for t,
    phi in degrees, tx, ty, decayed by `decay` per step) on the mean squared
    difference between warp(u, theta) and the target views (one loss per
    view, summed).  Every step runs in the library: the warp, the loss and its
    gradient (asift_warp_loss), the parameter gradients (asift_warp_bwd
    without the image gradient) and the update (asift_warp_adam).  Returns
    (theta history [steps+1, n, 4], loss history [steps+1, n])."""
    n = theta0.shape[0]
    theta = theta0.detach().clone().to(torch.float64).contiguous()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    tmax = lay.t_max if t_range[1] is None else t_range[1]
    lrs = (C.c_double * 4)(*[float(x) for x in lr])
    hist, losses = [theta.clone()], []
    for k in range(steps + 1):
        out = warp_forward(ctx, u, theta, lay)
        loss, vbar = warp_loss(ctx, out, target, lay, with_grad=k < steps)
        losses.append(loss)
        if k == steps:
            break
        _, g = warp_backward(ctx, u, theta, lay, vbar, image_grad=False)
        _check("asift_warp_adam", ctx.L.asift_warp_adam(ctx._ctx, n, _ptr(theta), _ptr(g), _ptr(m), _ptr(v), k, lrs,
                                                        float(decay), float(t_range[0]), float(tmax), _stream()))
        hist.append(theta.clone())
    return torch.stack(hist), torch.stack(losses)
