"""Thin Python binding of libsal.so (the C ABI in include/sal.h).

Argument marshalling only: every step of the saliency path runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  The functions keep the
C names (sal_create, sal_local_spectra_project, ...); `Saliency` is a small convenience
wrapper that owns a handle and allocates the outputs.

There is no CPU fallback: if libsal.so cannot be built or loaded, or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsal.so")

SAL_OK, SAL_ERR_INVALID_ARG, SAL_ERR_UNSUPPORTED, SAL_ERR_OOM, SAL_ERR_CUDA, SAL_ERR_TIMEOUT, \
    SAL_ERR_DEVICE_CHECK = range(7)
STATUS_NAMES = ["SAL_OK", "SAL_ERR_INVALID_ARG", "SAL_ERR_UNSUPPORTED", "SAL_ERR_OOM", "SAL_ERR_CUDA",
                "SAL_ERR_TIMEOUT", "SAL_ERR_DEVICE_CHECK"]
PRECISION = {"fp32": 0, "bf16": 1, "fp16": 2}
FEATURE = {"abs": 0, "energy": 1, "spatial": 2}   # E_m: mean over the cube's bins of |F_m| (step 3), of |F_m|^2,
#                                                   or over the cube's voxels of |IDFT(F_m)|
BOUNDARY = {"symmetric": 0, "periodic": 1, "zero": 2}
TAPER = {"rect": 0, "hann": 1}

# Exported entry points (must match include/sal.h).
ENTRY_POINTS = ("sal_create", "sal_destroy", "sal_workspace_size", "sal_set_alpha", "sal_local_spectra_project",
                "sal_center_surround", "sal_combine", "sal_saliency", "sal_saliency_backward", "sal_last_error",
                "sal_combine_noalloc", "sal_local_spectra_project_backward", "sal_center_surround_backward",
                "sal_combine_backward", "sal_launch_count", "sal_adapt_weights", "sal_directional_window",
                "sal_check_bounded_wait", "sal_measure_mufu_rate", "sal_measure_mma_rate")


class SalError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class sal_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("stride", ctypes.c_int), ("taper", ctypes.c_int),
                ("boundary", ctypes.c_int), ("feature", ctypes.c_int), ("n_offsets", ctypes.c_int),
                ("offsets", ctypes.POINTER(ctypes.c_int)), ("gauss_w", ctypes.POINTER(ctypes.c_float)),
                ("dir_id", ctypes.POINTER(ctypes.c_int)), ("n_dirs", ctypes.c_int),
                ("alpha", ctypes.POINTER(ctypes.c_float)), ("prec", ctypes.c_int),
                ("ls_delta", ctypes.c_double), ("hbm_budget_bytes", ctypes.c_size_t),
                ("n_directions", ctypes.c_int), ("directions", ctypes.POINTER(ctypes.c_int)),
                ("radius", ctypes.c_int), ("sigma", ctypes.c_double)]


class sal_adapt_params(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("mu", ctypes.c_double), ("eps", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("delta", ctypes.c_double), ("sections", ctypes.c_int)]


ADAPT_METHODS = {"lms": 0, "nlms": 1, "rls": 2}

_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libsal.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _build
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise SalError(SAL_ERR_UNSUPPORTED, f"{LIB_PATH} is missing (CUDA extension not built)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    L.sal_create.argtypes = [ctypes.POINTER(sal_params), i, i, i, ctypes.POINTER(vp)]
    L.sal_destroy.argtypes = [vp]
    L.sal_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.sal_set_alpha.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.sal_local_spectra_project.argtypes = [vp, vp, vp, vp]
    L.sal_center_surround.argtypes = [vp, vp, vp, vp]
    L.sal_combine.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.sal_saliency.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.sal_saliency_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.sal_combine_noalloc.argtypes = [i, i, i, vp, vp, vp, ctypes.c_double, vp, vp, vp]
    L.sal_local_spectra_project_backward.argtypes = [vp, vp, vp, vp, vp]
    L.sal_center_surround_backward.argtypes = [vp, vp, vp, vp, vp, vp]
    L.sal_combine_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.sal_launch_count.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
    L.sal_adapt_weights.argtypes = [vp, vp, vp, ctypes.POINTER(sal_adapt_params), vp, vp, vp]
    ip, fp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)
    L.sal_directional_window.argtypes = [i, ip, i, ctypes.c_double, i, ip, ip, fp, ip]
    L.sal_check_bounded_wait.argtypes = [vp, ctypes.c_uint, vp]
    L.sal_measure_mufu_rate.argtypes = [i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    L.sal_measure_mma_rate.argtypes = [i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    L.sal_last_error.argtypes = [vp]
    L.sal_last_error.restype = ctypes.c_char_p
    for name in ENTRY_POINTS:
        if name != "sal_last_error":
            getattr(L, name).restype = st
    _lib = L
    return L


def _check(status: int, handle=None):
    if status != SAL_OK:
        msg = load().sal_last_error(handle).decode()
        raise SalError(status, msg)


# ------------------------------------------------------------------------------------------------
# Parameters and the default directional window (Fig. 4: t, x and t-x directions)
# ------------------------------------------------------------------------------------------------

def directional_window(directions: Sequence[Sequence[int]] = ((1, 0, 0), (0, 1, 0), (1, 1, 0)), R: int = 3,
                       sigma: float = 1.5):
    """The library's directional window (sal_directional_window): neighbour offsets s*d for s in
    +-1..+-R along each direction d, their Gaussian factors and direction ids."""
    L = load()
    d = np.ascontiguousarray(directions, np.int32).reshape(-1, 3)
    cap = 64
    offs = np.zeros((cap, 3), np.int32)
    g = np.zeros(cap, np.float32)
    did = np.zeros(cap, np.int32)
    q = ctypes.c_int()
    ip = ctypes.POINTER(ctypes.c_int)
    _check(L.sal_directional_window(len(d), d.ctypes.data_as(ip), int(R), float(sigma), cap, ctypes.byref(q),
                                    offs.ctypes.data_as(ip), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                    did.ctypes.data_as(ip)), None)
    Q = q.value
    return offs[:Q].copy(), g[:Q].copy(), did[:Q].copy()


@dataclasses.dataclass
class Params:
    n: int = 16
    boundary: str = "symmetric"
    taper: str = "rect"
    directions: Tuple[Tuple[int, int, int], ...] = ((1, 0, 0), (0, 1, 0), (1, 1, 0))
    R: int = 3
    sigma: float = 1.5
    alpha: Optional[Sequence[float]] = None
    prec: str = "fp32"
    feature: str = "abs"
    stride: int = 1          # cubes at voxels whose indices are multiples of stride (1 < stride < n/2)
    ls_delta: float = 1e-6
    hbm_budget_bytes: int = 0
    offsets: Optional[np.ndarray] = None   # explicit window overrides directions/R/sigma
    gauss_w: Optional[np.ndarray] = None
    dir_id: Optional[np.ndarray] = None

    def n_dirs(self) -> int:
        if self.offsets is not None:
            did = np.asarray(self.dir_id)
            return int(did.max()) + 1 if did.size else 0
        return len(self.directions)


def sal_create(params: Params, shape: Sequence[int]):
    """Creates a handle on the current CUDA device and returns it.  Without an explicit window the
    library builds the directional window from params.directions, R and sigma."""
    L = load()
    ip, fp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)
    keep = []
    alpha = None if params.alpha is None else np.ascontiguousarray(params.alpha, np.float32)
    p = sal_params(n=params.n, stride=params.stride, taper=TAPER[params.taper], boundary=BOUNDARY[params.boundary],
                   feature=FEATURE[params.feature], prec=PRECISION[params.prec], ls_delta=params.ls_delta,
                   hbm_budget_bytes=params.hbm_budget_bytes)
    if params.offsets is not None:
        offs = np.ascontiguousarray(params.offsets, np.int32).reshape(-1, 3)
        g = np.ascontiguousarray(params.gauss_w, np.float32)
        did = np.ascontiguousarray(params.dir_id, np.int32)
        if alpha is None:
            alpha = np.ones(params.n_dirs(), np.float32)
        keep += [offs, g, did]
        p.n_offsets, p.offsets, p.gauss_w, p.dir_id = len(g), offs.ctypes.data_as(ip), g.ctypes.data_as(fp), \
            did.ctypes.data_as(ip)
        p.n_dirs = len(alpha)
    else:
        d = np.ascontiguousarray(params.directions, np.int32).reshape(-1, 3)
        keep.append(d)
        p.n_offsets, p.n_directions, p.directions = 0, len(d), d.ctypes.data_as(ip)
        p.radius, p.sigma = int(params.R), float(params.sigma)
    if alpha is not None:
        keep.append(alpha)
        p.alpha = alpha.ctypes.data_as(fp)
    h = ctypes.c_void_p()
    T, X, Y = (int(s) for s in shape)
    _check(L.sal_create(ctypes.byref(p), T, X, Y, ctypes.byref(h)), None)
    return h


def sal_destroy(h):
    if h:
        load().sal_destroy(h)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def sal_local_spectra_project(h, V, E, stream=None):
    _check(load().sal_local_spectra_project(h, _ptr(V), _ptr(E), _stream(stream)), h)


def sal_center_surround(h, E, S3, stream=None):
    _check(load().sal_center_surround(h, _ptr(E), _ptr(S3), _stream(stream)), h)


def sal_combine(h, S3, D, W_in, W_out, S, stream=None):
    _check(load().sal_combine(h, _ptr(S3), _ptr(D), _ptr(W_in), _ptr(W_out), _ptr(S), _stream(stream)), h)


def sal_saliency(h, V, D, W_in, S, S3_opt=None, E_opt=None, W_out=None, stream=None):
    _check(load().sal_saliency(h, _ptr(V), _ptr(D), _ptr(W_in), _ptr(S), _ptr(S3_opt), _ptr(E_opt), _ptr(W_out),
                               _stream(stream)), h)


def sal_saliency_backward(h, V, W, gS, gV=None, gW=None, galpha=None, stream=None):
    _check(load().sal_saliency_backward(h, _ptr(V), _ptr(W), _ptr(gS), _ptr(gV), _ptr(gW), _ptr(galpha),
                                        _stream(stream)), h)


def sal_local_spectra_project_backward(h, V, gE, gV, stream=None):
    _check(load().sal_local_spectra_project_backward(h, _ptr(V), _ptr(gE), _ptr(gV), _stream(stream)), h)


def sal_center_surround_backward(h, E, gS3, gE=None, galpha=None, stream=None):
    _check(load().sal_center_surround_backward(h, _ptr(E), _ptr(gS3), _ptr(gE), _ptr(galpha), _stream(stream)), h)


def sal_combine_backward(h, S3, W, gS, gS3, gW=None, stream=None):
    _check(load().sal_combine_backward(h, _ptr(S3), _ptr(W), _ptr(gS), _ptr(gS3), _ptr(gW), _stream(stream)), h)


def sal_combine_noalloc(S3, D, W_in, W_out, S, ls_delta: float = 1e-6, stream=None):
    """Allocation-free combination (no handle, no device allocation); S3 is [3][T][X][Y].  Runs on S3's
    device (made current for the call); every tensor must be float32, contiguous and on that device."""
    import torch
    if S3.dim() != 4 or S3.shape[0] != 3:
        raise SalError(SAL_ERR_INVALID_ARG, "S3 must be [3][T][X][Y]")
    shape = tuple(S3.shape[1:])
    want = {"S3": (S3, (3,) + shape), "S": (S, shape), "D": (D, shape), "W_in": (W_in, (3,)), "W_out": (W_out, (3,))}
    for name, (t, shp) in want.items():
        if t is None:
            if name in ("S3", "S"):
                raise SalError(SAL_ERR_INVALID_ARG, f"{name} must be given")
            continue
        if t.device != S3.device or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shp:
            raise SalError(SAL_ERR_INVALID_ARG, f"{name} must be a contiguous float32 tensor of shape {shp} on "
                                                f"{S3.device}")
    T, X, Y = (int(v) for v in shape)
    with torch.cuda.device(S3.device):
        st = stream if stream is not None else torch.cuda.current_stream(S3.device)
        _check(load().sal_combine_noalloc(T, X, Y, _ptr(S3), _ptr(D), _ptr(W_in), float(ls_delta), _ptr(W_out),
                                          _ptr(S), _stream(st)), None)


def sal_adapt_weights(h, S3, D, W_out, method: str = "nlms", sections: int = 0, mu: float = 0.5, eps: float = 1e-8,
                      lam: float = 1.0, delta: float = 1e-6, err2=None, stream=None):
    """The paper's sequential LMS / NLMS / RLS weight update on the GPU (one recursion per block of
    `sections` inline sections; 0 = whole volume).  W_out: device [blocks][3]."""
    p = sal_adapt_params(ADAPT_METHODS[method], float(mu), float(eps), float(lam), float(delta), int(sections))
    _check(load().sal_adapt_weights(h, _ptr(S3), _ptr(D), ctypes.byref(p), _ptr(W_out), _ptr(err2), _stream(stream)),
           h)


def sal_check_bounded_wait(h, tries: int = 1000, stream=None):
    """Makes one bounded mbarrier wait give up on purpose (failure-detection check): the next call on
    the handle returns SAL_ERR_TIMEOUT."""
    _check(load().sal_check_bounded_wait(h, int(tries), _stream(stream)), h)


def sal_measure_mufu_rate(op: str = "sqrt"):
    """Measured MUFU issue rate of the current device: (operations per second, SM count)."""
    r = ctypes.c_double()
    sms = ctypes.c_int()
    _check(load().sal_measure_mufu_rate({"sqrt": 0, "rsqrt": 1}[op], ctypes.byref(r), ctypes.byref(sms)), None)
    return float(r.value), int(sms.value)


def sal_measure_mma_rate(n_cols: int):
    """Measured cost of one tensor-core MMA (M = 128, K = 16) with n_cols columns on the current device:
    (SM cycles per MMA, SM count)."""
    r = ctypes.c_double()
    sms = ctypes.c_int()
    _check(load().sal_measure_mma_rate(int(n_cols), ctypes.byref(r), ctypes.byref(sms)), None)
    return float(r.value), int(sms.value)


def sal_launch_count() -> int:
    """Kernels launched by libsal.so in this process so far."""
    c = ctypes.c_ulonglong()
    _check(load().sal_launch_count(ctypes.byref(c)), None)
    return int(c.value)


def sal_set_alpha(h, alpha):
    a = np.ascontiguousarray(alpha, np.float32)
    _check(load().sal_set_alpha(h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), h)


def sal_workspace_size(h) -> int:
    b = ctypes.c_size_t()
    _check(load().sal_workspace_size(h, ctypes.byref(b)), h)
    return int(b.value)


class Saliency:
    """Owns a handle for one volume shape; allocates outputs with torch on the handle's device."""

    def __init__(self, shape: Sequence[int], params: Optional[Params] = None):
        import torch
        if not torch.cuda.is_available():
            raise SalError(SAL_ERR_CUDA, "no CUDA device: the saliency path runs only on the GPU")
        self.params = params or Params()
        self.shape = tuple(int(s) for s in shape)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.h = sal_create(self.params, self.shape)

    def close(self):
        if getattr(self, "h", None):
            sal_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, *lead):
        import torch
        return torch.empty(lead + self.shape, dtype=torch.float32, device=self.device)

    def _in(self, t):
        import torch
        if t is None:
            return None
        if not isinstance(t, torch.Tensor):
            t = torch.as_tensor(np.ascontiguousarray(t, np.float32))
        return t.to(self.device, torch.float32).contiguous()

    def local_spectra_project(self, V):
        E = self._empty(3)
        sal_local_spectra_project(self.h, self._in(V), E)
        return E

    def center_surround(self, E):
        S3 = self._empty(3)
        sal_center_surround(self.h, self._in(E), S3)
        return S3

    def combine(self, S3, D=None, W=None):
        import torch
        S = self._empty()
        W_out = torch.empty(3, dtype=torch.float32, device=self.device)
        sal_combine(self.h, self._in(S3), self._in(D), self._in(W), W_out, S)
        return S, W_out

    def saliency(self, V, D=None, W=None, intermediates: bool = False) -> Dict[str, "torch.Tensor"]:
        import torch
        S = self._empty()
        W_out = torch.empty(3, dtype=torch.float32, device=self.device)
        E = self._empty(3) if intermediates else None
        S3 = self._empty(3) if intermediates else None
        sal_saliency(self.h, self._in(V), self._in(D), self._in(W), S, S3, E, W_out)
        out = {"S": S, "W": W_out}
        if intermediates:
            out.update({"E": E, "S3": S3})
        return out

    def backward(self, V, W, gS):
        import torch
        gV = self._empty()
        gW = torch.empty(3, dtype=torch.float32, device=self.device)
        galpha = torch.empty(self.params.n_dirs(), dtype=torch.float32, device=self.device)
        sal_saliency_backward(self.h, self._in(V), self._in(W), self._in(gS), gV, gW, galpha)
        return gV, gW, galpha

    def set_alpha(self, alpha):
        sal_set_alpha(self.h, alpha)


def sal_last_error_text(h=None) -> str:
    """sal_last_error: message of the last error on the handle (or of the last sal_create)."""
    return load().sal_last_error(h).decode()
