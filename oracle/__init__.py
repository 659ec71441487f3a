"""FP64 CPU oracle of the local tone-mapping operator (arXiv 2102.01289).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` arm may import this
module. The product path (the CUDA library and its binding) never imports it,
and this module imports nothing from the product package.

The arithmetic lives in ``tm_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``); this file only builds and marshals it through ctypes.
Each function cites the equation of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libtmoracle.so")
_lock = threading.Lock()
_lib = None

MAX_FIELDS = 8
MAX_BINS = 256


def build(force: bool = False) -> str:
    """Compile ``tm_oracle.c`` into ``libtmoracle.so`` next to it (gcc, -O2)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tm_oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Mirror of ``tmo_params`` (paper notation: n, s, radii, eps, L_d, sat)."""

    _fields_ = [
        ("n_bins", ctypes.c_int32),
        ("n_fields", ctypes.c_int32),
        ("rx", ctypes.c_int32 * MAX_FIELDS),
        ("ry", ctypes.c_int32 * MAX_FIELDS),
        ("eps", ctypes.c_double * MAX_FIELDS),
        ("alpha", ctypes.c_double * MAX_FIELDS),
        ("ld_min", ctypes.c_double),
        ("ld_max", ctypes.c_double),
        ("sat", ctypes.c_double),
        ("flags", ctypes.c_int32),
    ]


# Reading variants (tm_oracle.h): Eq. 1 with <=, Algorithm 1's unclipped
# window area (zero padding), Eq. 10 on i / imax.
CDF_INCLUSIVE = 1
AREA_LITERAL = 2
VAR_LINEAR = 4


def make_params(n_bins: int, radii: Sequence, eps=0.1, alpha=1.0, ld_min=0.0,
                ld_max=1.0, sat=0.6, flags=0) -> Params:
    """Build oracle parameters. ``radii`` holds r or (rx, ry) per field.

    Defaults follow the paper: eps = 0.1 (Section II-C), sat = 0.6 (Eq. 12),
    alpha = 1 (plain Eq. 4), display range [0, 1] (Eq. 2, reading).
    """
    p = Params()
    p.n_bins = int(n_bins)
    p.n_fields = len(radii)
    for f, r in enumerate(radii):
        rx, ry = (r, r) if np.isscalar(r) else r
        p.rx[f], p.ry[f] = int(rx), int(ry)
        p.eps[f] = float(eps[f] if not np.isscalar(eps) else eps)
        p.alpha[f] = float(alpha[f] if not np.isscalar(alpha) else alpha)
    p.ld_min, p.ld_max, p.sat = float(ld_min), float(ld_max), float(sat)
    p.flags = int(flags)
    return p


def srgb_encode(c):
    """The sRGB transfer function (IEC 61966-2-1) on linear values in [0, 1]:
    12.92 c up to 0.0031308, 1.055 c^(1/2.4) - 0.055 above (FP64)."""
    c = np.clip(np.asarray(c, dtype=np.float64), 0.0, 1.0)
    return np.where(c <= 0.0031308, 12.92 * c, 1.055 * np.power(c, 1.0 / 2.4) - 0.055)


def to_u8(c, srgb=False):
    """uint8 output: floor(255 clamp(c, 0, 1) + 0.5), optionally sRGB-encoded first."""
    c = np.clip(np.asarray(c, dtype=np.float64), 0.0, 1.0)
    if srgb:
        c = srgb_encode(c)
    return np.floor(255.0 * c + 0.5).astype(np.uint8)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.tmo_luminance.restype = ctypes.c_float
            lib.tmo_luminance.argtypes = [ctypes.c_float] * 3
            lib.tmo_prepare.argtypes = [P, i32, i32, i32, P, P, P, P, P, P]
            lib.tmo_thresholds.argtypes = [ctypes.c_float, ctypes.c_float, i32, P]
            lib.tmo_integral_i64.argtypes = [P, i32, i32, P]
            lib.tmo_integral_f64.argtypes = [P, i32, i32, P]
            lib.tmo_integral_histogram.argtypes = [P, i32, i32, i32, P]
            lib.tmo_forward.argtypes = [P, i32, i32, P, P, P]
            lib.tmo_forward_range.argtypes = [P, i32, i32, P, P, P, P]
            lib.tmo_forward_pixels.argtypes = [P, i32, i32, P, P, P, i64, P, P, P, P, P, P]
            lib.tmo_forward_fixed_bins.argtypes = [P, i32, i32, P, P, P]
            lib.tmo_backward.argtypes = [P, i32, i32, P, i32, P, P, P, P]
            lib.tmo_window_counts.argtypes = [P, i32, i32, P, P]
            lib.tmo_merge_exposures.argtypes = [i32, P, P, i32, i32, P, P]
            lib.tmo_set_threads.argtypes = [i32]
            lib.tmo_num_procs.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _rgb32(rgb) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(rgb, dtype=np.float32))
    if a.ndim != 3 or a.shape[2] != 3:
        raise ValueError("rgb must be (H, W, 3)")
    return a


def luminance(r: float, g: float, b: float) -> float:
    """Eq. 11 in float, fixed order, floored at 1e-30f."""
    return float(_load().tmo_luminance(r, g, b))


def thresholds(imin: float, imax: float, n_bins: int) -> np.ndarray:
    """The n-1 bin edges of Section II-A as floats (rounded up)."""
    thr = np.zeros(max(n_bins - 1, 1), np.float32)
    _load().tmo_thresholds(ctypes.c_float(imin), ctypes.c_float(imax), n_bins, _ptr(thr))
    return thr[: n_bins - 1]


def prepare(rgb, n_bins: int) -> dict:
    """Eq. 11 luminance, global range, bin edges, bin map, normalised log."""
    a = _rgb32(rgb)
    H, W, _ = a.shape
    lum = np.empty((H, W), np.float32)
    bins = np.empty((H, W), np.uint8)
    lhat = np.empty((H, W), np.float64)
    thr = np.zeros(MAX_BINS, np.float32)
    imin = np.zeros(1, np.float32)
    imax = np.zeros(1, np.float32)
    rc = _load().tmo_prepare(_ptr(a), W, H, n_bins, _ptr(lum), _ptr(imin), _ptr(imax),
                             _ptr(thr), _ptr(bins), _ptr(lhat))
    if rc:
        raise ValueError(f"tmo_prepare failed ({rc})")
    return dict(lum=lum, imin=float(imin[0]), imax=float(imax[0]),
                thr=thr[: n_bins - 1].copy(), bins=bins, lhat=lhat)


def integral_i64(v) -> np.ndarray:
    """Eq. 5 over an int64 plane, modulo 2^64, with a zero first row/column."""
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
    H, W = a.shape
    S = np.empty((H + 1, W + 1), np.uint64)
    _load().tmo_integral_i64(_ptr(a), W, H, _ptr(S))
    return S


def integral_f64(v) -> np.ndarray:
    """Eq. 5 over a double plane, with a zero first row/column."""
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    H, W = a.shape
    S = np.empty((H + 1, W + 1), np.float64)
    _load().tmo_integral_f64(_ptr(a), W, H, _ptr(S))
    return S


def integral_histogram(bins, n_bins: int) -> np.ndarray:
    """Eq. 7-8: (n, H+1, W+1) uint32 integral images of the bin indicators."""
    a = np.ascontiguousarray(np.asarray(bins, dtype=np.uint8))
    H, W = a.shape
    Hk = np.empty((n_bins, H + 1, W + 1), np.uint32)
    _load().tmo_integral_histogram(_ptr(a), W, H, n_bins, _ptr(Hk))
    return Hk


def window_counts(bins, p: Params) -> np.ndarray:
    """Eq. 1 numerators alone, (s, H, W) uint32: the box sums (Eq. 9) of the
    integral image of [b(q) < b(p)] (Eq. 7-8 summed over the bins below)."""
    a = np.ascontiguousarray(np.asarray(bins, dtype=np.uint8))
    H, W = a.shape
    cnt = np.empty((p.n_fields, H, W), np.uint32)
    rc = _load().tmo_window_counts(_ptr(a), W, H, ctypes.byref(p), _ptr(cnt))
    if rc:
        raise ValueError(f"tmo_window_counts failed ({rc})")
    return cnt


def merge_exposures(ldr, times, log_response) -> np.ndarray:
    """Section III front-end (Debevec and Malik): the radiance map of n uint8
    (H, W, 3) exposures with exposure times ``times`` and the per-channel log
    inverse response ``log_response`` (3, 256). Returns (H, W, 3) float64."""
    imgs = [np.ascontiguousarray(np.asarray(a, dtype=np.uint8)) for a in ldr]
    H, W, _ = imgs[0].shape
    n = len(imgs)
    ptrs = (ctypes.c_void_p * n)(*[a.ctypes.data for a in imgs])
    t = np.ascontiguousarray(np.asarray(times, dtype=np.float64))
    g = np.ascontiguousarray(np.asarray(log_response, dtype=np.float64).reshape(3, 256))
    out = np.empty((H, W, 3), np.float64)
    rc = _load().tmo_merge_exposures(n, ctypes.cast(ptrs, ctypes.c_void_p), _ptr(t), W, H, _ptr(g), _ptr(out))
    if rc:
        raise ValueError(f"tmo_merge_exposures failed ({rc})")
    return out


def set_threads(n: int) -> None:
    """Host threads of the oracle's per-pixel loops (1 by default)."""
    _load().tmo_set_threads(int(n))


def num_procs() -> int:
    """Host cores the oracle's OpenMP runtime sees."""
    return int(_load().tmo_num_procs())


@dataclass
class Fields:
    cnt: np.ndarray
    area: np.ndarray
    mu: np.ndarray
    sigma2: np.ndarray
    weight: np.ndarray
    lf: np.ndarray
    l: np.ndarray


class _CFields(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("cnt", "area", "mu", "sigma2", "weight", "lf", "l")]


def forward(rgb, p: Params, range_=None):
    """Full forward (Eq. 11 -> Eq. 12). Returns (out (H,W,3) f64, Fields).
    range_: None, or (imin, imax) floats of an earlier frame to bin and
    normalise with (streaming reuse; the normalised log is clamped to [0, 1])."""
    a = _rgb32(rgb)
    H, W, _ = a.shape
    s = p.n_fields
    out = np.empty((H, W, 3), np.float64)
    fl = Fields(cnt=np.empty((s, H, W), np.uint32), area=np.empty((s, H, W), np.uint32),
                mu=np.empty((s, H, W)), sigma2=np.empty((s, H, W)), weight=np.empty((s, H, W)),
                lf=np.empty((s, H, W)), l=np.empty((H, W)))
    cf = _CFields(*[f.ctypes.data for f in (fl.cnt, fl.area, fl.mu, fl.sigma2, fl.weight, fl.lf, fl.l)])
    rng = None
    if range_ is not None:
        rng = np.ascontiguousarray(np.asarray(range_, dtype=np.float32))
    rc = _load().tmo_forward_range(_ptr(a), W, H, ctypes.byref(p), _ptr(rng) if rng is not None else None,
                                   _ptr(out), ctypes.byref(cf))
    if rc:
        raise ValueError(f"tmo_forward failed ({rc})")
    return out, fl


def forward_pixels(rgb, p: Params, xs, ys):
    """Forward at sampled pixels with every window statistic counted directly.

    Returns (out (K,3) f64, dict of cnt/area/sigma2/weight/lf each (K, s)).
    """
    a = _rgb32(rgb)
    H, W, _ = a.shape
    xs = np.ascontiguousarray(np.asarray(xs, dtype=np.int32))
    ys = np.ascontiguousarray(np.asarray(ys, dtype=np.int32))
    K, s = xs.shape[0], p.n_fields
    out = np.empty((K, 3), np.float64)
    d = dict(cnt=np.empty((K, s), np.uint32), area=np.empty((K, s), np.uint32),
             sigma2=np.empty((K, s)), weight=np.empty((K, s)), lf=np.empty((K, s)))
    rc = _load().tmo_forward_pixels(_ptr(a), W, H, ctypes.byref(p), _ptr(xs), _ptr(ys), K,
                                    _ptr(out), _ptr(d["cnt"]), _ptr(d["area"]),
                                    _ptr(d["sigma2"]), _ptr(d["weight"]), _ptr(d["lf"]))
    if rc:
        raise ValueError(f"tmo_forward_pixels failed ({rc})")
    return out, d


def forward_fixed_bins(rgb64, p: Params, bins) -> np.ndarray:
    """Smooth forward: double input, double luminance, bin map held fixed."""
    a = np.ascontiguousarray(np.asarray(rgb64, dtype=np.float64))
    H, W, _ = a.shape
    b = np.ascontiguousarray(np.asarray(bins, dtype=np.uint8))
    out = np.empty((H, W, 3), np.float64)
    rc = _load().tmo_forward_fixed_bins(_ptr(a), W, H, ctypes.byref(p), _ptr(b), _ptr(out))
    if rc:
        raise ValueError(f"tmo_forward_fixed_bins failed ({rc})")
    return out


def backward(rgb64, p: Params, grad_out, lum_f64: bool = False, bins=None):
    """FP64 adjoint with bins fixed. Returns (grad_in (H,W,3), grad_params dict)."""
    a = np.ascontiguousarray(np.asarray(rgb64, dtype=np.float64))
    H, W, _ = a.shape
    g = np.ascontiguousarray(np.asarray(grad_out, dtype=np.float64))
    s = p.n_fields
    gin = np.empty((H, W, 3), np.float64)
    gp = np.empty(3 + 2 * s, np.float64)
    bp = None
    if bins is not None:
        b = np.ascontiguousarray(np.asarray(bins, dtype=np.uint8))
        bp = _ptr(b)
    rc = _load().tmo_backward(_ptr(a), W, H, ctypes.byref(p), int(lum_f64), bp, _ptr(g),
                              _ptr(gin), _ptr(gp))
    if rc:
        raise ValueError(f"tmo_backward failed ({rc})")
    return gin, dict(ld_min=gp[0], ld_max=gp[1], sat=gp[2], eps=gp[3:3 + s].copy(),
                     alpha=gp[3 + s:3 + 2 * s].copy())
