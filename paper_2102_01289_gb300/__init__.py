"""Python binding of ``libtm.so``, the sm_103a local tone-mapping library.

Argument marshalling only: every step of the operator runs in the library's
CUDA kernels. PyTorch supplies device memory and streams. The functions keep
the C names (``tm_create``, ``tm_forward``, ``tm_backward``, ...). If the
library is missing, importing works but every call raises, so a missing build
is never silently replaced by another implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtm.so")

MAX_FIELDS = 8
MAX_BINS = 256

TM_OK, TM_EINVAL, TM_ENOMEM, TM_ECUDA, TM_EUNSUPPORTED, TM_ETIMEOUT, TM_ESTATE = range(7)
TM_F32, TM_F16, TM_U8 = 0, 1, 2
(TM_DBG_RANGE, TM_DBG_THRESHOLDS, TM_DBG_BINS, TM_DBG_Q, TM_DBG_COUNTS, TM_DBG_SIGMA2,
 TM_DBG_WEIGHT, TM_DBG_LF, TM_DBG_L, TM_DBG_QSHIFT) = range(1, 11)
TM_OPT_HIST_PATH = 1
TM_OPT_STAGE_TIMING = 2
TM_OPT_REUSE_RANGE = 3
TM_OPT_BACKWARD_REUSE = 4
TM_OPT_SWEEP_TILES = 5
TM_OPT_SWEEP_WIDTH = 6
# reading variants (tm_params.flags)
TM_FLAG_CDF_INCLUSIVE, TM_FLAG_AREA_LITERAL, TM_FLAG_VAR_LINEAR, TM_FLAG_SRGB_U8 = 1, 2, 4, 8

# Every symbol include/tm.h declares.
EXPORTS = (
    "tm_params_default", "tm_params_pyramid", "tm_create", "tm_destroy", "tm_last_error",
    "tm_status_string", "tm_forward", "tm_forward_host", "tm_forward_batch", "tm_backward",
    "tm_integral_image", "tm_integral_histogram", "tm_set_debug", "tm_debug_size",
    "tm_debug_export", "tm_set_option", "tm_last_launch_count", "tm_stage_times",
    "tm_integral_image_noalloc", "tm_backward_batch", "tm_forward_host_async", "tm_merge_exposures",
)


class TmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class TmParams(ctypes.Structure):
    _fields_ = [
        ("n_bins", ctypes.c_int32),
        ("n_fields", ctypes.c_int32),
        ("rx", ctypes.c_int32 * MAX_FIELDS),
        ("ry", ctypes.c_int32 * MAX_FIELDS),
        ("eps", ctypes.c_float * MAX_FIELDS),
        ("alpha", ctypes.c_float * MAX_FIELDS),
        ("ld_min", ctypes.c_float),
        ("ld_max", ctypes.c_float),
        ("sat", ctypes.c_float),
        ("flags", ctypes.c_int32),
    ]


class TmImage(ctypes.Structure):
    _fields_ = [
        ("data", ctypes.c_void_p),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("pitch", ctypes.c_int64),
        ("dtype", ctypes.c_int32),
    ]


_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import _build

    return _build.build(force=force)


def lib():
    """The loaded ``libtm.so``; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA extension first "
                               "(paper_2102_01289_gb300.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        st = ctypes.c_int
        sig = {
            "tm_params_default": (None, [P]),
            "tm_params_pyramid": (st, [P, i32, i32, i32, i32]),
            "tm_create": (st, [P, P]),
            "tm_destroy": (None, [P]),
            "tm_last_error": (ctypes.c_char_p, [P]),
            "tm_status_string": (ctypes.c_char_p, [st]),
            "tm_forward": (st, [P, P, P, P]),
            "tm_forward_host": (st, [P, P, P, P]),
            "tm_forward_batch": (st, [P, i32, P, P, P]),
            "tm_backward": (st, [P, P, P, P, P, P]),
            "tm_integral_image": (st, [P, i32, i32, P, P, P]),
            "tm_integral_histogram": (st, [P, i32, i32, i32, P, P]),
            "tm_set_debug": (st, [P, i32]),
            "tm_debug_size": (st, [P, i32, P]),
            "tm_debug_export": (st, [P, i32, P, sz, P]),
            "tm_set_option": (st, [P, i32, i64]),
            "tm_last_launch_count": (i64, [P]),
            "tm_stage_times": (i32, [P, P, P, i32]),
            "tm_integral_image_noalloc": (st, [P, i32, i32, P, P, P]),
            "tm_backward_batch": (st, [P, i32, P, P, P, P, P]),
            "tm_forward_host_async": (st, [P, P, P, P]),
            "tm_merge_exposures": (st, [i32, P, P, i32, i32, i64, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _status_name(s: int) -> str:
    try:
        return lib().tm_status_string(s).decode()
    except Exception:
        return f"status {s}"


def _check(status: int, ctx=None):
    if status != TM_OK:
        msg = lib().tm_last_error(ctx).decode(errors="replace")
        raise TmError(status, msg)


# ----------------------------------------------------------------- params --
def tm_params_default() -> TmParams:
    p = TmParams()
    lib().tm_params_default(ctypes.byref(p))
    return p


def tm_params_pyramid(width: int, height: int, n_fields: int, n_bins: int) -> TmParams:
    p = TmParams()
    _check(lib().tm_params_pyramid(ctypes.byref(p), width, height, n_fields, n_bins))
    return p


def make_params(n_bins: int, radii: Sequence, eps=0.1, alpha=1.0, ld_min=0.0, ld_max=1.0,
                sat=0.6, flags=0) -> TmParams:
    """Parameters from plain values; ``radii`` holds r or (rx, ry) per field."""
    p = tm_params_default()
    p.n_bins = int(n_bins)
    p.n_fields = len(radii)
    for f in range(MAX_FIELDS):
        if f < len(radii):
            r = radii[f]
            rx, ry = (r, r) if isinstance(r, (int,)) or not hasattr(r, "__len__") else r
            p.rx[f], p.ry[f] = int(rx), int(ry)
            p.eps[f] = float(eps if not hasattr(eps, "__len__") else eps[f])
            p.alpha[f] = float(alpha if not hasattr(alpha, "__len__") else alpha[f])
        else:
            p.rx[f] = p.ry[f] = 0
    p.ld_min, p.ld_max, p.sat = float(ld_min), float(ld_max), float(sat)
    p.flags = int(flags)
    return p


# ------------------------------------------------------------------ images --
def _dtype_code(t) -> int:
    import torch

    m = {torch.float32: TM_F32, torch.float16: TM_F16, torch.uint8: TM_U8}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def image_of(t) -> TmImage:
    """Descriptor of an (H, W, 3) tensor whose rows are dense RGB."""
    if t.dim() != 3 or t.shape[2] != 3:
        raise ValueError("image tensors are (H, W, 3)")
    if t.stride(2) != 1 or t.stride(1) != 3:
        raise ValueError("image rows must be dense interleaved RGB")
    return TmImage(t.data_ptr(), int(t.shape[1]), int(t.shape[0]), int(t.stride(0)), _dtype_code(t))


def image_of_numpy(a) -> TmImage:
    import numpy as np

    es = a.itemsize
    if (a.ndim != 3 or a.shape[2] != 3 or a.strides[2] != es or a.strides[1] != 3 * es
            or a.strides[0] % es or a.strides[0] < 3 * es * a.shape[1]):
        raise ValueError("host images are (H, W, 3) with contiguous pixels and rows (rows may be padded)")
    code = {np.dtype(np.float32): TM_F32, np.dtype(np.float16): TM_F16, np.dtype(np.uint8): TM_U8}[a.dtype]
    return TmImage(a.ctypes.data, a.shape[1], a.shape[0], a.strides[0] // es, code)


def _stream_ptr(stream) -> Optional[int]:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# -------------------------------------------------------------- entry points
def tm_create(params: TmParams):
    h = ctypes.c_void_p()
    _check(lib().tm_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def tm_destroy(ctx) -> None:
    if ctx:
        lib().tm_destroy(ctx)


def tm_last_error(ctx=None) -> str:
    return lib().tm_last_error(ctx).decode(errors="replace")


def tm_forward(ctx, inp, out, stream=None) -> None:
    a, b = image_of(inp), image_of(out)
    _check(lib().tm_forward(ctx, ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)), ctx)


def tm_forward_host(ctx, inp, out, stream=None) -> None:
    """Host (numpy) buffers in and out; copies and synchronisation inside."""
    a, b = image_of_numpy(inp), image_of_numpy(out)
    _check(lib().tm_forward_host(ctx, ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)), ctx)


def tm_forward_host_async(ctx, inp, out, stream=None) -> None:
    """Page-locked host (numpy) buffers in and out; enqueued on `stream`
    without synchronising (the upload overlaps the previous call's forward).
    Synchronise the stream before reading `out` or changing `inp`."""
    a, b = image_of_numpy(inp), image_of_numpy(out)
    _check(lib().tm_forward_host_async(ctx, ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)), ctx)


def tm_forward_batch(ctx, inputs, outputs, stream=None) -> None:
    n = len(inputs)
    if n != len(outputs):
        raise ValueError("inputs and outputs differ in length")
    A = (TmImage * max(n, 1))(*[image_of(t) for t in inputs])
    B = (TmImage * max(n, 1))(*[image_of(t) for t in outputs])
    _check(lib().tm_forward_batch(ctx, n, A, B, _stream_ptr(stream)), ctx)


def tm_backward(ctx, inp, grad_out, grad_in=None, grad_params=None, stream=None) -> None:
    a, g = image_of(inp), image_of(grad_out)
    gi = ctypes.byref(image_of(grad_in)) if grad_in is not None else None
    gp = grad_params.data_ptr() if grad_params is not None else None
    _check(lib().tm_backward(ctx, ctypes.byref(a), ctypes.byref(g), gi, gp, _stream_ptr(stream)), ctx)


def tm_backward_batch(ctx, inputs, grad_outs, grad_ins=None, grad_params=None, stream=None) -> None:
    """tm_backward over a list of images; grad_params receives the sum over them."""
    n = len(inputs)
    if n != len(grad_outs) or (grad_ins is not None and n != len(grad_ins)):
        raise ValueError("inputs, grad_outs and grad_ins differ in length")
    A = (TmImage * max(n, 1))(*[image_of(t) for t in inputs])
    G = (TmImage * max(n, 1))(*[image_of(t) for t in grad_outs])
    GI = (TmImage * max(n, 1))(*[image_of(t) for t in grad_ins]) if grad_ins is not None else None
    gp = grad_params.data_ptr() if grad_params is not None else None
    _check(lib().tm_backward_batch(ctx, n, A, G, GI, gp, _stream_ptr(stream)), ctx)


def tm_integral_image(q, s1, s2, stream=None) -> None:
    H, W = q.shape
    _check(lib().tm_integral_image(q.data_ptr(), W, H, s1.data_ptr(), s2.data_ptr(), _stream_ptr(stream)))


def tm_integral_image_noalloc(q, s1, s2, stream=None) -> None:
    """tm_integral_image for callers that must not allocate: its scratch is a
    static 8 MiB device array of the library (see include/tm.h)."""
    H, W = q.shape
    _check(lib().tm_integral_image_noalloc(q.data_ptr(), W, H, s1.data_ptr(), s2.data_ptr(),
                                           _stream_ptr(stream)))


def tm_merge_exposures(ldr, times, log_response, out, stream=None) -> None:
    """Section III capture front-end (Debevec and Malik): the radiance map of
    n uint8 (H, W, 3) device exposures with exposure times ``times`` (host
    floats) and the per-channel log inverse response ``log_response`` (3 x 256
    host floats), into the float32/float16 device image ``out``."""
    import numpy as np

    n = len(ldr)
    H, W = ldr[0].shape[:2]
    ptrs = (ctypes.c_void_p * n)(*[a.data_ptr() for a in ldr])
    t = (ctypes.c_float * n)(*[float(v) for v in times])
    g = (ctypes.c_float * 768)(*[float(v) for v in np.asarray(log_response, dtype=np.float64).reshape(-1)])
    o = image_of(out)
    _check(lib().tm_merge_exposures(n, ctypes.cast(ptrs, ctypes.c_void_p), ctypes.cast(t, ctypes.c_void_p), W, H,
                                    int(ldr[0].stride(0)), ctypes.cast(g, ctypes.c_void_p), ctypes.byref(o),
                                    _stream_ptr(stream)))


def tm_integral_histogram(bins, n_bins: int, hk, stream=None) -> None:
    H, W = bins.shape
    _check(lib().tm_integral_histogram(bins.data_ptr(), W, H, n_bins, hk.data_ptr(), _stream_ptr(stream)))


def tm_set_debug(ctx, enable: bool) -> None:
    _check(lib().tm_set_debug(ctx, int(bool(enable))), ctx)


def tm_set_option(ctx, key: int, value: int) -> None:
    _check(lib().tm_set_option(ctx, key, value), ctx)


def tm_last_launch_count(ctx) -> int:
    return int(lib().tm_last_launch_count(ctx))


def tm_stage_times(ctx) -> dict:
    """{stage name: summed milliseconds} since the previous read (syncs)."""
    cap = 16
    ms = (ctypes.c_float * cap)()
    names = (ctypes.c_char_p * cap)()
    n = lib().tm_stage_times(ctx, ms, names, cap)
    if n < 0:
        raise TmError(TM_ECUDA, tm_last_error(ctx))
    return {names[i].decode(): float(ms[i]) for i in range(n)}


def tm_debug_export(ctx, what: int, stream=None):
    """Copy one debug plane into a new device tensor (dtype per include/tm.h)."""
    import torch

    n = ctypes.c_size_t()
    _check(lib().tm_debug_size(ctx, what, ctypes.byref(n)), ctx)
    dt = {TM_DBG_BINS: torch.uint8, TM_DBG_Q: torch.int32, TM_DBG_COUNTS: torch.int32,
          TM_DBG_QSHIFT: torch.int32}.get(what, torch.float32)
    elem = torch.tensor([], dtype=dt).element_size()
    dst = torch.empty(max(n.value // elem, 1), dtype=dt, device="cuda")
    _check(lib().tm_debug_export(ctx, what, dst.data_ptr(), n.value, _stream_ptr(stream)), ctx)
    return dst[: n.value // elem]


def params_tensor(p: TmParams):
    """[ld_min, ld_max, sat, eps[0..s-1], alpha[0..s-1]] as a float32 CPU tensor
    (the layout tm_backward's grad_params uses)."""
    import torch

    s = p.n_fields
    vals = [p.ld_min, p.ld_max, p.sat] + [p.eps[f] for f in range(s)] + [p.alpha[f] for f in range(s)]
    return torch.tensor(vals, dtype=torch.float32)


def params_from_tensor(template: TmParams, t) -> TmParams:
    """Parameters of `template` with the differentiable values taken from t."""
    p = TmParams.from_buffer_copy(template)
    v = [float(x) for x in t.detach().cpu().reshape(-1)]
    s = p.n_fields
    p.ld_min, p.ld_max, p.sat = v[0], v[1], v[2]
    for f in range(s):
        p.eps[f] = v[3 + f]
        p.alpha[f] = v[3 + s + f]
    return p


class _CtxCache:
    """tm_ctx per distinct parameter values (the C context copies them)."""

    def __init__(self, template: TmParams):
        self.template = template
        self.ctxs = {}

    def get(self, t):
        key = tuple(round(float(x), 9) for x in t.detach().cpu().reshape(-1))
        if key not in self.ctxs:
            c = tm_create(params_from_tensor(self.template, t))
            # the autograd function keeps its input saved and unchanged between
            # forward and backward, so the backward may take the forward's
            # intermediates from the context (it checks they are that input's)
            tm_set_option(c, TM_OPT_BACKWARD_REUSE, 1)
            self.ctxs[key] = c
        return self.ctxs[key]

    def close(self):
        for c in self.ctxs.values():
            tm_destroy(c)
        self.ctxs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


try:
    import torch as _torch

    class TMFunction(_torch.autograd.Function):
        """Differentiable tone mapping: forward through tm_forward (a batch
        through tm_forward_batch), backward through the hand-written adjoint
        tm_backward / tm_backward_batch (bins held fixed).

        Inputs: img (H, W, 3) or (B, H, W, 3) float32 CUDA tensor; theta, the
        float32 parameter vector of params_tensor(); cache, a _CtxCache.
        Returns the tone-mapped image (float32)."""

        @staticmethod
        def forward(ctx, img, theta, cache):
            c = cache.get(theta)
            x = img.contiguous()
            out = _torch.empty_like(x)
            if x.dim() == 3:
                tm_forward(c, x, out)
            else:
                tm_forward_batch(c, [x[b] for b in range(x.shape[0])], [out[b] for b in range(x.shape[0])])
            ctx.save_for_backward(x, theta)
            ctx.cache = cache
            return out

        @staticmethod
        def backward(ctx, grad_out):
            x, theta = ctx.saved_tensors
            c = ctx.cache.get(theta)
            g = grad_out.contiguous().float()
            gin = _torch.empty_like(x) if ctx.needs_input_grad[0] else None
            gp = _torch.empty(theta.numel(), dtype=_torch.float32, device=x.device)
            if x.dim() == 3:
                tm_backward(c, x, g, gin, gp)
            else:
                B = x.shape[0]
                tm_backward_batch(c, [x[b] for b in range(B)], [g[b] for b in range(B)],
                                  [gin[b] for b in range(B)] if gin is not None else None, gp)
            gtheta = gp.to(theta.device) if ctx.needs_input_grad[1] else None
            return gin, gtheta, None

except ImportError:  # pragma: no cover
    TMFunction = None


class ToneMapper:
    """Owns a ``tm_ctx``; ``forward`` runs the whole operator on a device image."""

    def __init__(self, params: TmParams):
        self.params = params
        self.ctx = tm_create(params)

    def forward(self, x, out=None, out_dtype=None, stream=None):
        import torch

        if out is None:
            out = torch.empty(x.shape, dtype=out_dtype or x.dtype, device=x.device)
        tm_forward(self.ctx, x, out, stream)
        return out

    __call__ = forward

    def close(self):
        if self.ctx:
            tm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
