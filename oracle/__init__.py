"""CPU oracle for the ASIFT-view + ORB + Hamming-matching hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline / reference
leg may import this package.  The product library never calls it, and it shares
no code with the CUDA path.  The arithmetic lives in ``asift_oracle.c`` (plain
scalar C, fp64 warp, integer ORB and matching); this module compiles it with gcc
on first use and wraps it with ctypes, plus a plain-Python driver that chains the
per-view steps in the paper's order (views -> ORB -> pooled matching).

Every function cites the passage it follows in ``asift_oracle.c``.  Parity status:
all functions are pinned by tests/test_oracle_pins.py (closed forms, exact special
cases, library routines, brute force).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "asift_oracle.c"), os.path.join(_HERE, "sift_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

N_BINS = 30
N_PAIRS = 256
PATTERN_SEED = 250303479


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OView(C.Structure):
    _fields_ = [("k", C.c_int32), ("j", C.c_int32), ("W", C.c_int32), ("H", C.c_int32),
                ("Wr", C.c_int32), ("Hr", C.c_int32), ("Wv", C.c_int32), ("Hv", C.c_int32),
                ("K", C.c_int32), ("pad", C.c_int32),
                ("t", C.c_double), ("phi_deg", C.c_double), ("sigma", C.c_double), ("scale", C.c_double),
                ("cq", C.c_int64), ("sq", C.c_int64), ("tq", C.c_int64)]


class ODView(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("Wr", C.c_int32), ("Hr", C.c_int32),
                ("Wv", C.c_int32), ("Hv", C.c_int32), ("K", C.c_int32), ("pad", C.c_int32),
                ("t", C.c_double), ("phi", C.c_double), ("tx", C.c_double), ("ty", C.c_double)]


SIFT_KP_DTYPE = np.dtype([("x", np.float64), ("y", np.float64), ("sigma", np.float64), ("angle", np.float64),
                          ("response", np.float64), ("octave", np.int32), ("layer", np.int32)])

KP_DTYPE = np.dtype([("x", np.int16), ("y", np.int16), ("level", np.uint8), ("bin", np.uint8),
                     ("pad", np.int16), ("r25", np.int64)])

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
        kpp = np.ctypeslib.ndpointer(KP_DTYPE, flags="C_CONTIGUOUS")
        L.oracle_sizeof_view.restype = C.c_int
        L.oracle_sizeof_kp.restype = C.c_int
        assert L.oracle_sizeof_view() == C.sizeof(OView)
        assert L.oracle_sizeof_kp() == KP_DTYPE.itemsize
        L.oracle_view_table.argtypes = [C.c_int, C.c_int, C.c_int, P(OView), C.c_int]
        L.oracle_view_table.restype = C.c_int
        L.oracle_gauss_taps.argtypes = [C.c_double, C.c_int, f64p]
        L.oracle_lanczos3.argtypes = [C.c_double]
        L.oracle_lanczos3.restype = C.c_double
        L.oracle_lanczos3_weights.argtypes = [C.c_double, f64p]
        L.oracle_warp_view.argtypes = [u8p, C.c_int, P(OView), C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_warp_view_f64.argtypes = [f64p, C.c_int, P(OView), C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_warp_view_nn.argtypes = [u8p, C.c_int, P(OView), C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_lanczos.argtypes = [C.c_double, C.c_int]
        L.oracle_lanczos.restype = C.c_double
        L.oracle_lanczos_weights.argtypes = [C.c_double, C.c_int, f64p]
        L.oracle_warp_view_lanczos.argtypes = [u8p, C.c_int, P(OView), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_warp_view_lanczos_f64.argtypes = [f64p, C.c_int, P(OView), C.c_int, C.c_void_p, C.c_void_p,
                                                   C.c_void_p]
        L.oracle_warp_view_nn_f64.argtypes = [f64p, C.c_int, P(OView), C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_make_view.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, P(OView)]
        L.oracle_make_view_scaled.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, P(OView)]
        L.oracle_view_table_scaled.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, P(OView), C.c_int]
        L.oracle_view_table_scaled.restype = C.c_int
        L.oracle_level_size.argtypes = [C.c_int, C.c_int]
        L.oracle_level_size.restype = C.c_int
        L.oracle_downscale.argtypes = [u8p, C.c_void_p, C.c_int, C.c_int, u8p, C.c_void_p, C.c_int, C.c_int]
        L.oracle_smooth.argtypes = [u8p, C.c_int, C.c_int, u8p]
        L.oracle_fast9.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.oracle_fast9.restype = C.c_int
        L.oracle_harris25.argtypes = [u8p, C.c_int, C.c_int, C.c_int]
        L.oracle_harris25.restype = C.c_int64
        L.oracle_detect_level.argtypes = [u8p, u8p, C.c_int, C.c_int, C.c_int, i32p, i32p, i64p, C.c_int]
        L.oracle_detect_level.restype = C.c_int
        L.oracle_quota.argtypes = [i32p, i32p, C.c_int, C.c_int, i32p]
        L.oracle_bin_table.argtypes = [i64p]
        L.oracle_angle_bin.argtypes = [C.c_int64, C.c_int64]
        L.oracle_angle_bin.restype = C.c_int
        L.oracle_moments.argtypes = [u8p, C.c_int, C.c_int, C.c_int, P(C.c_int64), P(C.c_int64)]
        L.oracle_pattern.argtypes = [C.c_uint64, i8p]
        L.oracle_brief.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_int, i8p, u8p]
        L.oracle_orb_view.argtypes = [u8p, u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, i8p,
                                      kpp, u8p, C.c_int]
        L.oracle_orb_view.restype = C.c_int
        L.oracle_match.argtypes = [u8p, C.c_int, u8p, C.c_int, C.c_int, C.c_int, i32p, i32p, i32p, u8p]
        L.oracle_match.restype = C.c_int
        L.oracle_sizeof_dview.restype = C.c_int
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        L.oracle_dedup.argtypes = [f32p, f32p, f32p, f32p, C.c_int, u8p]
        L.oracle_dedup.restype = C.c_int
        L.oracle_reproj_sq.argtypes = [f64p, C.c_double, C.c_double, C.c_double, C.c_double]
        L.oracle_reproj_sq.restype = C.c_double
        L.oracle_precision_count.argtypes = [f32p, f32p, f32p, f32p, C.c_int, f64p, C.c_double]
        L.oracle_precision_count.restype = C.c_int
        L.oracle_homography4.argtypes = [f64p, f64p, f64p, f64p, f64p]
        L.oracle_homography4.restype = C.c_int
        L.oracle_ransac.argtypes = [f32p, f32p, f32p, f32p, C.c_int, u32p, C.c_int, C.c_double, i32p, f64p, u8p]
        L.oracle_ransac.restype = C.c_int
        L.oracle_scale_coefficient.argtypes = [f32p, f32p, f32p, f32p, i32p, C.c_int]
        L.oracle_scale_coefficient.restype = C.c_double
        L.oracle_gauss_blur.argtypes = [f64p, C.c_int, C.c_int, C.c_double, f64p]
        L.oracle_sift.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        L.oracle_sift.restype = C.c_int
        L.oracle_sift_ex.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, f64p, f64p, C.c_int,
                                     P(C.c_int), C.c_double]
        L.oracle_sift_ex.restype = C.c_int
        L.oracle_sift_match.argtypes = [f32p, C.c_int, f32p, C.c_int, C.c_double, i32p, f64p, f64p, u8p]
        L.oracle_sift_match_f32.argtypes = [f32p, C.c_int, f32p, C.c_int, C.c_double, i32p, f32p, f32p, u8p]
        L.oracle_sizeof_sift_kp.restype = C.c_int
        assert L.oracle_sizeof_sift_kp() == SIFT_KP_DTYPE.itemsize
        assert L.oracle_sizeof_dview() == C.sizeof(ODView)
        L.oracle_dwarp_fwd.argtypes = [f64p, P(ODView), f64p]
        L.oracle_dwarp_vjp.argtypes = [f64p, P(ODView), f64p, f64p, f64p]
        L.oracle_backproject.argtypes = [P(OView), C.c_int, C.c_double, C.c_double,
                                         P(C.c_double), P(C.c_double)]
        _lib = L
    return _lib


# ---------------------------------------------------------------- view table
def view_table(H: int, W: int, kmax: int) -> list[OView]:
    """Sec. III-B sampling rule: t = sqrt(2)^k (k <= kmax), phi = j 72/t deg < 180."""
    n = lib().oracle_view_table(H, W, kmax, None, 0)
    arr = (OView * n)()
    lib().oracle_view_table(H, W, kmax, arr, n)
    return list(arr)


def make_view(H: int, W: int, t: float, phi_deg: float, scale: float = 1.0) -> OView:
    """A view descriptor for any tilt t >= 1, longitude phi (degrees) and
    scale s > 0 (Eq. (2)'s S: the canvas magnifies the source by s)."""
    v = OView()
    lib().oracle_make_view_scaled(H, W, float(t), float(phi_deg), float(scale), C.byref(v))
    return v


def view_table_scaled(H: int, W: int, kmax: int, ds: float) -> list[OView]:
    """The coarse stage's parameter groups (Sec. III-B): the (t, phi) list with
    the scale s = 1 + k ds tied to the tilt exponent k."""
    n = lib().oracle_view_table_scaled(H, W, kmax, float(ds), None, 0)
    arr = (OView * n)()
    lib().oracle_view_table_scaled(H, W, kmax, float(ds), arr, n)
    return list(arr)


def gauss_taps(sigma: float, K: int) -> np.ndarray:
    g = np.zeros(K + 1, dtype=np.float64)
    lib().oracle_gauss_taps(sigma, K, g)
    return g


def lanczos3(x: float) -> float:
    """Eq. (4) with a = 3."""
    return lib().oracle_lanczos3(float(x))


def lanczos3_weights(f: float) -> np.ndarray:
    w = np.zeros(6, dtype=np.float64)
    lib().oracle_lanczos3_weights(float(f), w)
    return w


# ---------------------------------------------------------------- warp
@dataclass
class ViewOut:
    f64: np.ndarray
    u8: np.ndarray
    mask: np.ndarray


def warp_view(u: np.ndarray, v: OView) -> ViewOut:
    """Eq. (2)-(4): rotation (Lanczos-3) -> Gaussian along x -> tilt (Lanczos-3).

    ``u`` is uint8 or float64 (H, W)."""
    H, W = u.shape
    assert (H, W) == (v.H, v.W)
    f = np.zeros((v.Hv, v.Wv), dtype=np.float64)
    b = np.zeros((v.Hv, v.Wv), dtype=np.uint8)
    m = np.zeros((v.Hv, v.Wv), dtype=np.uint8)
    if u.dtype == np.uint8:
        u = np.ascontiguousarray(u)
        lib().oracle_warp_view(u, W, C.byref(v), f.ctypes.data, b.ctypes.data, m.ctypes.data)
    else:
        u = np.ascontiguousarray(u, dtype=np.float64)
        lib().oracle_warp_view_f64(u, W, C.byref(v), f.ctypes.data, b.ctypes.data, m.ctypes.data)
    return ViewOut(f, b, m)


def warp_view_nn(u: np.ndarray, v: OView) -> ViewOut:
    """The nearest-neighbour form of the coarse stage (Sec. III-B): nearest
    source pixel for the rotation, Gaussian along x, nearest canvas column for
    the tilt.  ``u`` is uint8 or float64 (H, W)."""
    H, W = u.shape
    assert (H, W) == (v.H, v.W)
    f = np.zeros((v.Hv, v.Wv), dtype=np.float64)
    b = np.zeros((v.Hv, v.Wv), dtype=np.uint8)
    m = np.zeros((v.Hv, v.Wv), dtype=np.uint8)
    if u.dtype == np.uint8:
        u = np.ascontiguousarray(u)
        lib().oracle_warp_view_nn(u, W, C.byref(v), f.ctypes.data, b.ctypes.data, m.ctypes.data)
    else:
        u = np.ascontiguousarray(u, dtype=np.float64)
        lib().oracle_warp_view_nn_f64(u, W, C.byref(v), f.ctypes.data, b.ctypes.data, m.ctypes.data)
    return ViewOut(f, b, m)


def lanczos(x: float, a: int) -> float:
    """Eq. (4): L(x; a)."""
    return lib().oracle_lanczos(float(x), int(a))


def lanczos_weights(f: float, a: int) -> np.ndarray:
    """Normalised Eq. (3) weights of taps floor(p) - a + 1 .. floor(p) + a."""
    w = np.zeros(2 * a)
    lib().oracle_lanczos_weights(float(f), int(a), w)
    return w


def warp_view_lanczos(u: np.ndarray, v: OView, a: int) -> ViewOut:
    """The view with Lanczos-a resampling (a = 4: the precise stage's 8 x 8
    reproduction of the best view, Sec. III-C)."""
    assert 1 <= a <= 8
    H, W = u.shape
    assert (H, W) == (v.H, v.W)
    f = np.zeros((v.Hv, v.Wv), dtype=np.float64)
    b = np.zeros((v.Hv, v.Wv), dtype=np.uint8)
    m = np.zeros((v.Hv, v.Wv), dtype=np.uint8)
    if u.dtype == np.uint8:
        u = np.ascontiguousarray(u)
        lib().oracle_warp_view_lanczos(u, W, C.byref(v), a, f.ctypes.data, b.ctypes.data, m.ctypes.data)
    else:
        u = np.ascontiguousarray(u, dtype=np.float64)
        lib().oracle_warp_view_lanczos_f64(u, W, C.byref(v), a, f.ctypes.data, b.ctypes.data, m.ctypes.data)
    return ViewOut(f, b, m)


# ---------------------------------------------------------------- ORB pieces
def level_size(n0: int, l: int) -> int:
    return lib().oracle_level_size(n0, l)


def downscale(src: np.ndarray, msk: np.ndarray | None, Wl: int, Hl: int):
    src = np.ascontiguousarray(src, dtype=np.uint8)
    Hp, Wp = src.shape
    dst = np.zeros((Hl, Wl), dtype=np.uint8)
    mdst = np.zeros((Hl, Wl), dtype=np.uint8)
    if msk is None:
        lib().oracle_downscale(src, None, Wp, Hp, dst, None, Wl, Hl)
        return dst
    msk = np.ascontiguousarray(msk, dtype=np.uint8)
    lib().oracle_downscale(src, msk.ctypes.data, Wp, Hp, dst, mdst.ctypes.data, Wl, Hl)
    return dst, mdst


def pyramid(view: np.ndarray, mask: np.ndarray, L: int):
    levels, masks = [np.ascontiguousarray(view)], [np.ascontiguousarray(mask)]
    H0, W0 = view.shape
    for l in range(1, L):
        d, m = downscale(levels[-1], masks[-1], level_size(W0, l), level_size(H0, l))
        levels.append(d)
        masks.append(m)
    return levels, masks


def smooth(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.zeros_like(img)
    lib().oracle_smooth(img, W, H, out)
    return out


def fast9(img: np.ndarray, x: int, y: int, thr: int = 20) -> bool:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    return bool(lib().oracle_fast9(img, img.shape[1], x, y, thr))


def harris25(img: np.ndarray, x: int, y: int) -> int:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    return int(lib().oracle_harris25(img, img.shape[1], x, y))


def detect_level(img: np.ndarray, mask: np.ndarray, thr: int = 20, cap: int = 1 << 22):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    H, W = img.shape
    cap = min(cap, H * W)
    xs = np.zeros(cap, np.int32)
    ys = np.zeros(cap, np.int32)
    rs = np.zeros(cap, np.int64)
    n = lib().oracle_detect_level(img, mask, W, H, thr, xs, ys, rs, cap)
    return xs[:n].copy(), ys[:n].copy(), rs[:n].copy()


def quota(Ws, Hs, N: int) -> np.ndarray:
    L = len(Ws)
    q = np.zeros(L, np.int32)
    lib().oracle_quota(np.asarray(Ws, np.int32), np.asarray(Hs, np.int32), L, N, q)
    return q


def bin_table() -> np.ndarray:
    e = np.zeros((N_BINS, 2), np.int64)
    lib().oracle_bin_table(e)
    return e


def angle_bin(mx: int, my: int) -> int:
    return lib().oracle_angle_bin(int(mx), int(my))


def moments(img: np.ndarray, x: int, y: int):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    a, b = C.c_int64(), C.c_int64()
    lib().oracle_moments(img, img.shape[1], x, y, C.byref(a), C.byref(b))
    return a.value, b.value


def pattern(seed: int = PATTERN_SEED) -> np.ndarray:
    pat = np.zeros((N_BINS, N_PAIRS, 4), np.int8)
    lib().oracle_pattern(seed, pat)
    return pat


def brief(sm: np.ndarray, x: int, y: int, b: int, pat: np.ndarray) -> np.ndarray:
    sm = np.ascontiguousarray(sm, dtype=np.uint8)
    d = np.zeros(32, np.uint8)
    lib().oracle_brief(sm, sm.shape[1], x, y, b, np.ascontiguousarray(pat), d)
    return d


@dataclass
class OrbOut:
    kps: np.ndarray      # KP_DTYPE, canonical order (level, then selection order)
    desc: np.ndarray     # (n, 32) uint8


def orb_view(view: np.ndarray, mask: np.ndarray, L: int, N: int, thr: int = 20,
             pat: np.ndarray | None = None, cand_cap: int = 1 << 22) -> OrbOut:
    """ORB [23] on one view: pyramid, FAST-9/Harris/NMS, quota, centroid, steered BRIEF."""
    view = np.ascontiguousarray(view, dtype=np.uint8)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    if pat is None:
        pat = pattern()
    H, W = view.shape
    kps = np.zeros(max(N, 1), KP_DTYPE)
    desc = np.zeros((max(N, 1), 32), np.uint8)
    n = lib().oracle_orb_view(view, mask, W, H, L, N, thr, np.ascontiguousarray(pat), kps, desc,
                              min(cand_cap, W * H))
    if n < 0:
        raise RuntimeError(f"oracle candidate capacity exceeded at level {-1 - n}")
    return OrbOut(kps[:n].copy(), desc[:n].copy())


# ---------------------------------------------------------------- matching
@dataclass
class MatchOut:
    best: np.ndarray
    d1: np.ndarray
    d2: np.ndarray
    accepted: np.ndarray


def match(q: np.ndarray, t: np.ndarray, num: int = 4, den: int = 5) -> MatchOut:
    """Brute-force Hamming matcher with the nearest/second-nearest ratio test."""
    q = np.ascontiguousarray(q, dtype=np.uint8).reshape(-1, 32)
    t = np.ascontiguousarray(t, dtype=np.uint8).reshape(-1, 32)
    nq, nt = len(q), len(t)
    best = np.zeros(max(nq, 1), np.int32)
    d1 = np.zeros(max(nq, 1), np.int32)
    d2 = np.zeros(max(nq, 1), np.int32)
    acc = np.zeros(max(nq, 1), np.uint8)
    if nq:
        lib().oracle_match(q, nq, t if nt else np.zeros((1, 32), np.uint8), nt, num, den, best, d1, d2, acc)
    return MatchOut(best[:nq], d1[:nq], d2[:nq], acc[:nq].astype(bool))


def backproject(v: OView, level: int, xl: float, yl: float):
    sx, sy = C.c_double(), C.c_double()
    lib().oracle_backproject(C.byref(v), level, xl, yl, C.byref(sx), C.byref(sy))
    return sx.value, sy.value


# ---------------------------------------------------------------- whole pair
@dataclass
class PoolOut:
    kps: np.ndarray       # KP_DTYPE, all views, canonical order
    view_of: np.ndarray   # view index of each keypoint
    desc: np.ndarray
    src_xy: np.ndarray    # (n, 2) back-projected source coordinates


def image_pool(img: np.ndarray, kmax: int, L: int, N: int, thr: int = 20,
               pat: np.ndarray | None = None, views=None, view_outs=None) -> PoolOut:
    """All simulated views of one image -> ORB per view -> pooled keypoints."""
    if pat is None:
        pat = pattern()
    H, W = img.shape
    if views is None:
        views = view_table(H, W, kmax)
    kl, vl, dl, xy = [], [], [], []
    for vi, v in enumerate(views):
        vo = view_outs[vi] if view_outs is not None else warp_view(img, v)
        o = orb_view(vo.u8, vo.mask, L, N, thr, pat)
        kl.append(o.kps)
        dl.append(o.desc)
        vl.append(np.full(len(o.kps), vi, np.int32))
        xy.append(np.array([backproject(v, int(k["level"]), float(k["x"]), float(k["y"])) for k in o.kps],
                           dtype=np.float64).reshape(-1, 2))
    return PoolOut(np.concatenate(kl), np.concatenate(vl), np.concatenate(dl), np.concatenate(xy))


def match_pair(img1: np.ndarray, img2: np.ndarray, kmax: int, L: int, N: int, thr: int = 20,
               num: int = 4, den: int = 5):
    """The whole hot path for one pair: pooled views of both images, matched."""
    pat = pattern()
    p1 = image_pool(img1, kmax, L, N, thr, pat)
    p2 = image_pool(img2, kmax, L, N, thr, pat)
    m = match(p1.desc, p2.desc, num, den)
    return p1, p2, m


# ---------------------------------------------------------------- differentiable warp
def dview(H: int, W: int, t0: float, phi0: float, K: int, t=None, phi=None, tx=0.0, ty=0.0) -> ODView:
    """Fixed sizes from (t0, phi0) (as the view table would give them), current
    parameters (t, phi, tx, ty)."""
    base = make_view(H, W, t0, phi0)
    v = ODView()
    v.W, v.H, v.Wr, v.Hr, v.Wv, v.Hv, v.K = W, H, base.Wr, base.Hr, base.Wv, base.Hv, K
    v.t = t0 if t is None else t
    v.phi = phi0 if phi is None else phi
    v.tx, v.ty = tx, ty
    return v


def dwarp_fwd(u: np.ndarray, v: ODView) -> np.ndarray:
    """Differentiable warp: clamped Lanczos-3 rotation, Gaussian, tilt (fp64)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros((v.Hv, v.Wv), np.float64)
    lib().oracle_dwarp_fwd(u, C.byref(v), out)
    return out


def dwarp_vjp(u: np.ndarray, v: ODView, vbar: np.ndarray):
    """Exact transpose of dwarp_fwd: (ubar, [tbar, phibar, txbar, tybar])."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    vbar = np.ascontiguousarray(vbar, dtype=np.float64)
    ub = np.zeros_like(u)
    pb = np.zeros(4, np.float64)
    lib().oracle_dwarp_vjp(u, C.byref(v), vbar, ub, pb)
    return ub, pb


# ---------------------------------------------------------------- evaluation on the accepted pairs
def _xy(pairs):
    """(x1, y1, x2, y2) float32 arrays of a pair list (structured array with those fields,
    or an (n, 4) array)."""
    if getattr(pairs, "dtype", None) is not None and pairs.dtype.names:
        cols = [pairs[f] for f in ("x1", "y1", "x2", "y2")]
    else:
        a = np.asarray(pairs, dtype=np.float32).reshape(-1, 4)
        cols = [a[:, k] for k in range(4)]
    return [np.ascontiguousarray(c, dtype=np.float32) for c in cols]


def dedup(pairs) -> np.ndarray:
    """Keep mask: a pair is kept iff no earlier pair has the same nearest pixels
    of (x1, y1, x2, y2) (duplicate correspondences from several views)."""
    x1, y1, x2, y2 = _xy(pairs)
    keep = np.zeros(len(x1), np.uint8)
    lib().oracle_dedup(x1, y1, x2, y2, len(x1), keep)
    return keep.astype(bool)


def reproj_sq(H: np.ndarray, x: float, y: float, u: float, v: float) -> float:
    return lib().oracle_reproj_sq(np.ascontiguousarray(H, np.float64).reshape(9), x, y, u, v)


def precision_count(pairs, H: np.ndarray, th_sq: float = 3.0) -> int:
    """Eq. (6): pairs within sqrt(th_sq) of the true mapping (R_Num of Eq. (5))."""
    x1, y1, x2, y2 = _xy(pairs)
    return lib().oracle_precision_count(x1, y1, x2, y2, len(x1), np.ascontiguousarray(H, np.float64).reshape(9),
                                        th_sq)


def homography4(src: np.ndarray, dst: np.ndarray):
    """H (3x3, h8 = 1) from 4 correspondences src[k] -> dst[k], or None when degenerate."""
    src, dst = np.asarray(src, np.float64), np.asarray(dst, np.float64)
    H = np.zeros(9)
    ok = lib().oracle_homography4(np.ascontiguousarray(src[:, 0]), np.ascontiguousarray(src[:, 1]),
                                  np.ascontiguousarray(dst[:, 0]), np.ascontiguousarray(dst[:, 1]), H)
    return H.reshape(3, 3) if ok else None


@dataclass
class RansacOut:
    best: int
    counts: np.ndarray      # int32 per hypothesis (-1: repeated pair or degenerate fit)
    Hs: np.ndarray          # (n_hyp, 9)
    inlier: np.ndarray      # bool per pair


def ransac(pairs, rnd: np.ndarray, th_sq: float = 9.0) -> RansacOut:
    """RANSAC [28] with the random numbers given: rnd is uint32 (n_hyp, 4)."""
    x1, y1, x2, y2 = _xy(pairs)
    rnd = np.ascontiguousarray(rnd, dtype=np.uint32).reshape(-1, 4)
    n_hyp = len(rnd)
    counts = np.zeros(n_hyp, np.int32)
    Hs = np.zeros(9 * n_hyp)
    inl = np.zeros(len(x1), np.uint8)
    best = lib().oracle_ransac(x1, y1, x2, y2, len(x1), rnd.reshape(-1), n_hyp, th_sq, counts, Hs, inl)
    return RansacOut(best, counts, Hs.reshape(n_hyp, 9), inl.astype(bool))


def scale_coefficient(pairs, des=None) -> float:
    """Eq. (1): the scaling coefficient f from image 1 to image 2 over the pairs
    in list order; des: per-pair descriptor distances (default: the pairs'
    'd1' field, the nearest Hamming distance)."""
    x1, y1, x2, y2 = _xy(pairs)
    if des is None:
        des = pairs["d1"]
    des = np.ascontiguousarray(des, dtype=np.int32)
    return lib().oracle_scale_coefficient(x1, y1, x2, y2, des, len(x1))


# ---------------------------------------------------------------- SIFT (the precise stage's detector)
def gauss_blur(u: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian, radius int(4 sigma + 0.5), normalised taps, edge pixels replicated."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    H, W = u.shape
    out = np.zeros_like(u)
    lib().oracle_gauss_blur(u, W, H, float(sigma), out)
    return out


@dataclass
class SiftOut:
    kps: np.ndarray          # SIFT_KP_DTYPE
    desc: np.ndarray         # float32 (n, 128), unit L2 norm


def sift(img: np.ndarray, max_kp: int = 5000) -> SiftOut:
    """Lowe's SIFT on an 8-bit image: the strongest max_kp keypoints and their descriptors."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    kps = np.zeros(max_kp, SIFT_KP_DTYPE)
    desc = np.zeros((max_kp, 128), np.float32)
    n = lib().oracle_sift(img, W, H, max_kp, kps.ctypes.data, desc.ctypes.data)
    return SiftOut(kps[:n].copy(), desc[:n].copy())


@dataclass
class SiftMarginOut:
    kps: np.ndarray
    desc: np.ndarray
    margin: np.ndarray       # per keypoint: smallest relative margin of its decisions
    miss: np.ndarray         # (m, 4): candidates rejected by <= M relative: x, y, sigma, angle (-1: any)


def sift_margins(img: np.ndarray, max_kp: int = 20000, M: float = 2e-3, max_miss: int = 100000) -> SiftMarginOut:
    """sift() plus, for parity tests, each keypoint's smallest decision margin
    and the near-miss candidates (rejected by at most M relative)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    kps = np.zeros(max_kp, SIFT_KP_DTYPE)
    desc = np.zeros((max_kp, 128), np.float32)
    margin = np.zeros(max_kp, np.float64)
    miss = np.zeros((max_miss, 4), np.float64)
    nm = C.c_int(0)
    n = lib().oracle_sift_ex(img, W, H, max_kp, kps.ctypes.data, desc.ctypes.data, margin, miss.reshape(-1), max_miss,
                             C.byref(nm), float(M))
    return SiftMarginOut(kps[:n].copy(), desc[:n].copy(), margin[:n].copy(), miss[:nm.value].copy())


@dataclass
class SiftMatchOut:
    best: np.ndarray
    d1: np.ndarray           # squared L2 distances
    d2: np.ndarray
    accepted: np.ndarray


def sift_match(q: np.ndarray, t: np.ndarray, ratio: float = 0.8) -> SiftMatchOut:
    q = np.ascontiguousarray(q, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    nq, nt = len(q), len(t)
    best = np.zeros(nq, np.int32)
    d1 = np.zeros(nq)
    d2 = np.zeros(nq)
    acc = np.zeros(nq, np.uint8)
    lib().oracle_sift_match(q.reshape(-1) if nq else np.zeros(1, np.float32), nq,
                            t.reshape(-1) if nt else np.zeros(1, np.float32), nt, float(ratio), best, d1, d2, acc)
    return SiftMatchOut(best, d1, d2, acc.astype(bool))


def sift_match_f32(q: np.ndarray, t: np.ndarray, ratio: float = 0.8) -> SiftMatchOut:
    """Brute-force L2 SIFT matching with the ratio test, decisions in fp32 in the
    fixed order of sift_oracle.c (the precision the GPU decides in); d1, d2 are
    the fp32 squared distances."""
    q = np.ascontiguousarray(q, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    nq, nt = len(q), len(t)
    best = np.zeros(max(nq, 1), np.int32)
    d1 = np.zeros(max(nq, 1), np.float32)
    d2 = np.zeros(max(nq, 1), np.float32)
    acc = np.zeros(max(nq, 1), np.uint8)
    if nq:
        lib().oracle_sift_match_f32(q.reshape(-1), nq, t.reshape(-1) if nt else np.zeros(1, np.float32), nt,
                                    float(ratio), best, d1, d2, acc)
    return SiftMatchOut(best[:nq], d1[:nq], d2[:nq], acc[:nq].astype(bool))

