"""FP64 CPU oracle of the seismic saliency method (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
import this package.  It shares no code with the CUDA path: the stencil builder,
the normalisation, the weight fits and the gradients below are written here from
the paper, independently of the product.

Pipeline (Sec. 2 of the paper, Fig. 2 block diagram):
  V --local 3D DFT (Eq. 2)--> F --projection (Eq. 1)--> F_m --abs mean (step 3)--> E_m
    --directional center-surround (Eq. 3)--> S_m --min-max--> S^_m
    --weighted sum (Eq. 4; equal, given, LS fit to a desired map D, or LMS/NLMS/RLS)--> S.

Readings where the paper is silent (each an argument here):
  * stride 1 (a window around every voxel), window offsets [-n/2, n/2-1]; stride s < n/2 (windows
    overlapping by more than half) as an option, with E interpolated (trilinear) between the lattice
    voxels and held constant past the last lattice point of an axis;
  * rectangular taper (the cube C_n as is); Hann optional;
  * E_m = (1/n^3) sum_{k != 0} r_m(k) |F[k]| (feature "abs"); the energy reading of the garbled step 3,
    E_m = (1/n^3) sum_{k != 0} r_m(k)^2 |F[k]|^2, is feature "energy"; its spatial-domain reading,
    the mean over the cube of |IDFT(F_m)|, is `spatial_features`;
  * DCS stencil: direction groups t, x and t-x (Fig. 4), offsets s*d for s in +-1..+-R,
    Gaussian weights w_o = alpha_d exp(-|o|^2 / (2 sigma^2)) multiplying the neighbour
    inside |.| as Eq. 3 is written, Q = number of offsets;
  * borders: symmetric extension (edge sample repeated) of V and of E;
  * per-map min-max before combining and a final min-max of S (a flat map is all 0);
  * LS weights (G + delta I)^-1 b in FP64 (the fixed point the LMS family approaches;
    RLS with lambda = 1 and P0 = I/delta reaches it exactly).
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

BOUNDARY = {"symmetric": 0, "periodic": 1, "zero": 2}
TAPER = {"rect": 0, "hann": 1}
FEATURE = {"abs": 0, "energy": 1}   # step 3: mean of |F_m| (the paper's), or of |F_m|^2

_lib = None
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_i64_p = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L_ = ctypes.c_long
        i = ctypes.c_int
        L.sal_oracle_local_spectrum.argtypes = [_c_dbl_p, L_, L_, L_, i, i, i, L_, L_, L_, _c_dbl_p]
        L.sal_oracle_projected_spectra.argtypes = [_c_dbl_p, L_, L_, L_, i, i, i, L_, L_, L_, _c_dbl_p]
        L.sal_oracle_features.argtypes = [_c_dbl_p, L_, L_, L_, i, i, i, i, _c_dbl_p, i]
        L.sal_oracle_features_at.argtypes = [_c_dbl_p, L_, L_, L_, i, i, i, i, _c_i64_p, L_, _c_dbl_p, i]
        L.sal_oracle_center_surround.argtypes = [_c_dbl_p, L_, L_, L_, i, i, _c_int_p, _c_dbl_p, _c_dbl_p, i]
        L.sal_oracle_center_surround_adjoint.argtypes = [_c_dbl_p, L_, L_, L_, i, i, _c_int_p, _c_dbl_p,
                                                         _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.sal_oracle_features_adjoint.argtypes = [_c_dbl_p, L_, L_, L_, i, i, i, i, _c_dbl_p, _c_dbl_p, i]
        L.sal_oracle_band_count.argtypes = [_c_dbl_p, L_, L_, L_, i, i, i, ctypes.c_double, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int32), i]
        L.sal_oracle_lms.argtypes = [_c_dbl_p, _c_dbl_p, L_, ctypes.c_double, _c_dbl_p, _c_dbl_p]
        L.sal_oracle_nlms.argtypes = [_c_dbl_p, _c_dbl_p, L_, ctypes.c_double, ctypes.c_double, _c_dbl_p,
                                      _c_dbl_p]
        L.sal_oracle_rls.argtypes = [_c_dbl_p, _c_dbl_p, L_, ctypes.c_double, ctypes.c_double, _c_dbl_p,
                                     _c_dbl_p]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_c_dbl_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed (code {rc})")


# ----------------------------------------------------------------------------------------------
# Steps 1-3: local spectrum, projection, features (Eq. 1, Eq. 2, step 3)
# ----------------------------------------------------------------------------------------------

def local_spectrum(V, t: int, x: int, y: int, n: int, boundary="symmetric", taper="rect") -> np.ndarray:
    """Complex [n][n][n] spectrum of the cube around voxel (t,x,y) (Eq. 2)."""
    V = _f64(V)
    out = np.empty((n, n, n, 2), dtype=np.float64)
    _check(lib().sal_oracle_local_spectrum(_dp(V), *V.shape, n, BOUNDARY[boundary], TAPER[taper],
                                           t, x, y, _dp(out)), "local_spectrum")
    return out[..., 0] + 1j * out[..., 1]


def projected_spectra(V, t: int, x: int, y: int, n: int, boundary="symmetric", taper="rect") -> np.ndarray:
    """Complex [3][n][n][n] projected spectra F_t, F_x, F_y of Eq. 1 (DC = 0)."""
    V = _f64(V)
    out = np.empty((3, n, n, n, 2), dtype=np.float64)
    _check(lib().sal_oracle_projected_spectra(_dp(V), *V.shape, n, BOUNDARY[boundary], TAPER[taper],
                                              t, x, y, _dp(out)), "projected_spectra")
    return out[..., 0] + 1j * out[..., 1]


def features(V, n: int, boundary="symmetric", taper="rect", threads: int = 0, feature="abs",
             stride: int = 1) -> np.ndarray:
    """E [3][T][X][Y] (E_t, E_x, E_y) at every voxel: the mean over the cube's bins of |F_m|
    (feature "abs", step 3) or of |F_m|^2 (feature "energy").  stride s > 1: the cubes sit only on
    the lattice of voxels whose indices are all multiples of s (windows overlapping by n - s of n,
    the paper's ">50% overlap" for s < n/2), and E elsewhere is interpolated from them (upsample).
    Feature "spatial": the mean over the cube of |IDFT(F_m)| (spatial_features; stride 1)."""
    V = _f64(V)
    if feature == "spatial":
        if stride != 1:
            raise ValueError("the spatial-domain reading is defined here for stride 1")
        return spatial_features(V, n, boundary, taper)
    if stride > 1:
        T, X, Y = V.shape
        lat = [np.arange(0, d, stride) for d in (T, X, Y)]
        pts = np.stack(np.meshgrid(*lat, indexing="ij"), -1).reshape(-1, 3)
        Ec = features_at(V, pts, n, boundary, taper, threads, feature).T.reshape((3,) + tuple(len(a) for a in lat))
        return upsample(Ec, stride, V.shape)
    E = np.empty((3,) + V.shape, dtype=np.float64)
    _check(lib().sal_oracle_features(_dp(V), *V.shape, n, BOUNDARY[boundary], TAPER[taper], FEATURE[feature],
                                     _dp(E), threads), "features")
    return E


def spatial_features_at(V, pts, n: int, boundary="symmetric", taper="rect") -> np.ndarray:
    """The spatial-domain reading of the feature step at listed voxels, pts [count][3] -> [count][3]:
    E_m = (1/n^3) sum_u |f_m[u]|, f_m the inverse DFT over the cube of the projected spectrum F_m of Eq. 1
    (DC = 0).  f_m is real up to rounding: F is Hermitian for a real cube and the ratio P_m / |k| depends
    on squared signed indices only.  Projected spectra from `projected_spectra`, then numpy's inverse FFT
    (a library step); one voxel at a time, for small cases."""
    pts = np.asarray(pts, dtype=np.int64).reshape(-1, 3)
    out = np.empty((pts.shape[0], 3), dtype=np.float64)
    for i, (t, x, y) in enumerate(pts.tolist()):
        f = np.fft.ifftn(projected_spectra(V, t, x, y, n, boundary, taper), axes=(1, 2, 3))
        out[i] = np.abs(f).mean(axis=(1, 2, 3))
    return out


def spatial_features(V, n: int, boundary="symmetric", taper="rect") -> np.ndarray:
    """E [3][T][X][Y] of the spatial-domain reading at every voxel (spatial_features_at over the volume)."""
    shape = np.asarray(V).shape
    pts = np.stack(np.meshgrid(*[np.arange(d) for d in shape], indexing="ij"), -1).reshape(-1, 3)
    return spatial_features_at(V, pts, n, boundary, taper).T.reshape((3,) + shape)


def _eq1_ratios(n: int) -> np.ndarray:
    """r_m(k) = P_m(k) / |k| of Eq. 1 over the n^3 bins (signed indices; zero at DC): [3][n][n][n]."""
    s = np.array([k if k < n // 2 else k - n for k in range(n)], dtype=np.float64)
    i, j, k = np.meshgrid(s, s, s, indexing="ij")
    r = np.sqrt(i * i + j * j + k * k)
    P = np.stack([np.sqrt(j * j + k * k), np.sqrt(i * i + k * k), np.sqrt(i * i + j * j)])
    return np.where(r > 0, P / np.where(r > 0, r, 1.0), 0.0)


def _taper3(n: int, taper: str) -> np.ndarray:
    u = np.arange(n)
    h = np.ones(n) if taper == "rect" else 0.5 - 0.5 * np.cos(2.0 * np.pi * u / n)
    return h[:, None, None] * h[None, :, None] * h[None, None, :]


def spatial_features_adjoint(V, gE, n: int, boundary="symmetric", taper="rect") -> np.ndarray:
    """gV = (dE/dV)^T gE for the spatial-domain reading.  Per voxel p, with w the tapered window and
    A_m = IDFT diag(r_m) DFT (a real circulant, symmetric since r_m is even in k): f_m = A_m w and
    E_m = (1/n^3) sum_u |f_m[u]|, so dE_m/dw = (1/n^3) A_m sign(f_m) (sign(0) = 0); each window's
    gradient, times the taper, goes back to the voxels its samples came from through the border
    extension.  numpy's FFTs as library steps; small cases only."""
    V = _f64(V)
    gE = _f64(gE)
    T, X, Y = V.shape
    R = _eq1_ratios(n)
    h3 = _taper3(n, taper)
    gV = np.zeros_like(V)
    off = np.arange(n) - n // 2
    for t in range(T):
        for x in range(X):
            for y in range(Y):
                it, ix, iy = (ext_index(c + off, N, boundary) for c, N in ((t, T), (x, X), (y, Y)))
                ok = (it[:, None, None] >= 0) & (ix[None, :, None] >= 0) & (iy[None, None, :] >= 0)
                w = np.where(ok, V[np.ix_(np.maximum(it, 0), np.maximum(ix, 0), np.maximum(iy, 0))], 0.0) * h3
                F = np.fft.fftn(w)
                gw = np.zeros((n, n, n))
                for m in range(3):
                    f = np.real(np.fft.ifftn(R[m] * F))
                    gw += gE[m, t, x, y] * np.real(np.fft.ifftn(R[m] * np.fft.fftn(np.sign(f))))
                gw *= h3 / n ** 3
                np.add.at(gV, np.ix_(np.maximum(it, 0), np.maximum(ix, 0), np.maximum(iy, 0)), np.where(ok, gw, 0.0))
    return gV


def upsample_adjoint(gE, stride: int) -> np.ndarray:
    """Transpose of `upsample`: every voxel's gradient goes back to the two lattice points of each axis
    it was interpolated from, with the same weights (1 - f, f; 1 past the last lattice point)."""
    out = _f64(gE)
    for ax in range(3):
        N = out.shape[ax + 1]
        L = -(-N // stride)
        res = np.zeros(out.shape[:ax + 1] + (L,) + out.shape[ax + 2:])
        for i in range(N):
            a = i // stride
            f = (i - a * stride) / stride
            val = np.take(out, i, axis=ax + 1)
            lo = [slice(None)] * res.ndim
            lo[ax + 1] = a
            if a + 1 < L:
                hi = list(lo)
                hi[ax + 1] = a + 1
                res[tuple(lo)] += (1.0 - f) * val
                res[tuple(hi)] += f * val
            else:
                res[tuple(lo)] += val
        out = res
    return out


def upsample(Ec, stride: int, shape) -> np.ndarray:
    """Lattice values Ec [3][Tc][Xc][Yc] (at indices multiples of s) to every voxel of `shape`:
    along each axis, a voxel between lattice points a = s floor(i/s) and a + s takes the linear
    interpolation (1 - f) E(a) + f E(a + s), f = (i - a)/s; past the last lattice point of the axis
    it takes that point's value.  Applied axis by axis (trilinear)."""
    out = _f64(Ec)
    for ax, N in enumerate(shape):
        L = out.shape[ax + 1]
        res = np.empty(out.shape[:ax + 1] + (N,) + out.shape[ax + 2:])
        for i in range(N):
            a = i // stride
            f = (i - a * stride) / stride
            lo = np.take(out, a, axis=ax + 1)
            if a + 1 < L:
                hi = np.take(out, a + 1, axis=ax + 1)
                val = (1.0 - f) * lo + f * hi
            else:
                val = lo
            idx = [slice(None)] * res.ndim
            idx[ax + 1] = i
            res[tuple(idx)] = val
        out = res
    return out


def features_at(V, pts, n: int, boundary="symmetric", taper="rect", threads: int = 0,
                feature="abs") -> np.ndarray:
    """E at listed voxels: pts [count][3] -> [count][3]."""
    if feature == "spatial":
        return spatial_features_at(V, pts, n, boundary, taper)
    V = _f64(V)
    pts = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    out = np.empty((pts.shape[0], 3), dtype=np.float64)
    if pts.shape[0] == 0:
        return out
    _check(lib().sal_oracle_features_at(_dp(V), *V.shape, n, BOUNDARY[boundary], TAPER[taper], FEATURE[feature],
                                        pts.ctypes.data_as(_c_i64_p), pts.shape[0], _dp(out), threads),
           "features_at")
    return out


# Kink band of the |F| adjoint: a bin counts as F = 0 when |F| <= ZERO_BIN * ||window||_1.  The
# level is set by FP64 arithmetic (an exactly zero bin comes out of the FP64 DFT below 2^-45 of the
# window L1 norm for n <= 32).
ZERO_BIN = 2.0 ** -40
# Windows holding a bin with ZERO_BIN < |F| / L1 <= ILL_BIN are ill-conditioned for the adjoint of
# step 3: its direction F / |F| is known to FP32 arithmetic only to about 2^-24 L1 / |F| (and the
# FP32 forms zero bins below 2^-19 L1), so a few such bins move the gradient of a small volume by
# more than 1e-5.  4 x 2^-19 = 2^-17.
ILL_BIN = 2.0 ** -17


def band_count(V, n: int, boundary="symmetric", taper="rect", lo: float = ZERO_BIN, hi: float = ILL_BIN,
               threads: int = 0) -> np.ndarray:
    """Per voxel [T][X][Y]: the number of non-DC bins of its cube with lo < |F| / L1 <= hi, L1 the
    window's L1 norm (test helper for the conditioning of the feature adjoint)."""
    V = _f64(V)
    out = np.empty(V.shape, dtype=np.int32)
    _check(lib().sal_oracle_band_count(_dp(V), *V.shape, n, BOUNDARY[boundary], TAPER[taper], lo, hi,
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), threads),
           "band_count")
    return out


def adjoint_footprint(flags, n: int, boundary="symmetric") -> np.ndarray:
    """Voxels whose feature-adjoint gradient receives a term from a flagged window: the cube
    p + u - n/2 (u in [0, n)^3) of every flagged p, folded back through the border extension."""
    flags = np.asarray(flags, bool)
    T, X, Y = flags.shape
    out = np.zeros(flags.shape, bool)
    for t, x, y in zip(*np.nonzero(flags)):
        a, b, c = (ext_index(np.arange(n) + p - n // 2, N, boundary) for p, N in ((t, T), (x, X), (y, Y)))
        a, b, c = a[a >= 0], b[b >= 0], c[c >= 0]
        out[np.ix_(a, b, c)] = True
    return out


# ----------------------------------------------------------------------------------------------
# 2-D sections (one inline or crossline section A [X][Y]: the method with square n x n windows)
# ----------------------------------------------------------------------------------------------

def section_features(A, n: int, boundary="symmetric") -> np.ndarray:
    """Per-pixel features of a 2-D section A [X][Y] with n x n windows (offsets -n/2 .. n/2-1, border
    extension as for volumes): F = 2-D DFT of the window, signed bins (j, k); Eq. 1 in two dimensions
    keeps, for each axis, the frequency component of the other axis: r_x = |k| / |(j, k)|,
    r_y = |j| / |(j, k)|; E_x, E_y = (1/n^2) sum over bins != 0 of r |F|.  Returned with the
    unprojected mean (1/n^2) sum |F| in front: [E_0, E_x, E_y] [3][X][Y]."""
    A = _f64(A)
    X, Y = A.shape
    mode = {"symmetric": "symmetric", "periodic": "wrap", "zero": "constant"}[boundary]
    P = np.pad(A, n, mode=mode)
    sb = np.where(np.arange(n) < n // 2, np.arange(n), np.arange(n) - n).astype(np.float64)
    j, k = np.meshgrid(sb, sb, indexing="ij")
    rad = np.sqrt(j * j + k * k)
    rad[0, 0] = 1.0
    r = np.stack([np.ones((n, n)), np.abs(k) / rad, np.abs(j) / rad])
    r[:, 0, 0] = 0.0
    E = np.empty((3, X, Y))
    for x in range(X):
        for y in range(Y):
            w = P[x + n - n // 2: x + n - n // 2 + n, y + n - n // 2: y + n - n // 2 + n]
            mag = np.abs(np.fft.fft2(w))
            for m in range(3):
                E[m, x, y] = np.sum(r[m] * mag) / (n * n)
    return E


def section_saliency(A, n: int, boundary="symmetric", directions=((0, 1, 0), (0, 0, 1), (0, 1, 1)), R: int = 3,
                     sigma: float = 1.5, weights=(0.0, 0.5, 0.5)) -> Dict[str, np.ndarray]:
    """The method on a 2-D section: section features, an in-plane directional center-surround (Eq. 3)
    and the combination of the two projected maps (Eq. 4; the unprojected map gets weight 0)."""
    E2 = section_features(A, n, boundary)[:, None]          # [3][1][X][Y]
    offs, g, did, w = dcs_stencil(directions, R, sigma)
    S3 = center_surround(E2, offs, w, boundary)
    out = combine(S3, np.asarray(weights, float))
    out.update({"E": E2, "S3": S3})
    return out


# ----------------------------------------------------------------------------------------------
# Step 4: directional center-surround (Eq. 3, Fig. 4)
# ----------------------------------------------------------------------------------------------

DEFAULT_DIRECTIONS = ((1, 0, 0), (0, 1, 0), (1, 1, 0))  # t, x and t-x (Fig. 4)


def dcs_stencil(directions: Sequence[Sequence[int]] = DEFAULT_DIRECTIONS, R: int = 3, sigma: float = 1.5,
                alpha: Optional[Sequence[float]] = None):
    """Directional window: offsets o = s*d (s = +-1..+-R) per direction d, Gaussian factor
    g_o = exp(-|o|^2 / (2 sigma^2)), weight w_o = alpha_d g_o.  Returns
    (offsets [Q][3] int32, g [Q], dir_id [Q] int32, w [Q])."""
    alpha = np.ones(len(directions)) if alpha is None else np.asarray(alpha, dtype=np.float64)
    offs, g, did = [], [], []
    for d_i, d in enumerate(directions):
        for s in list(range(-R, 0)) + list(range(1, R + 1)):
            o = (s * d[0], s * d[1], s * d[2])
            offs.append(o)
            g.append(math.exp(-(o[0] ** 2 + o[1] ** 2 + o[2] ** 2) / (2.0 * sigma * sigma)))
            did.append(d_i)
    offs = np.asarray(offs, dtype=np.int32)
    g = np.asarray(g, dtype=np.float64)
    did = np.asarray(did, dtype=np.int32)
    return offs, g, did, alpha[did] * g


def center_surround(E, offsets, w, boundary="symmetric", threads: int = 0) -> np.ndarray:
    """S [3][T][X][Y] per Eq. 3 (raw, before normalisation)."""
    E = _f64(E)
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    w = _f64(w)
    S = np.empty_like(E)
    _check(lib().sal_oracle_center_surround(_dp(E), *E.shape[1:], BOUNDARY[boundary], len(w),
                                            offsets.ctypes.data_as(_c_int_p), _dp(w), _dp(S), threads),
           "center_surround")
    return S


def ext_index(i, N: int, boundary: str):
    """Boundary extension of one axis (array version); -1 where the zero extension applies."""
    i = np.asarray(i, dtype=np.int64)
    if boundary == "periodic":
        return np.mod(i, N)
    if boundary == "zero":
        return np.where((i >= 0) & (i < N), i, -1)
    r = np.mod(i, 2 * N)
    return np.where(r < N, r, 2 * N - 1 - r)


def center_surround_at(V, pts, n: int, offsets, w, boundary="symmetric", taper="rect",
                       threads: int = 0, feature="abs") -> Tuple[np.ndarray, np.ndarray]:
    """(E at pts [count][3], raw S at pts [count][3]) computed from V one voxel at a time."""
    pts = np.asarray(pts, dtype=np.int64).reshape(-1, 3)
    shape = np.asarray(V).shape
    offsets = np.asarray(offsets, dtype=np.int64)
    nb = pts[:, None, :] + offsets[None, :, :]                 # [count][Q][3]
    idx = np.stack([ext_index(nb[..., a], shape[a], boundary) for a in range(3)], axis=-1)
    valid = np.all(idx >= 0, axis=-1)
    allp = np.concatenate([pts, np.where(valid[..., None], idx, 0).reshape(-1, 3)], axis=0)
    uniq, inv = np.unique(allp, axis=0, return_inverse=True)
    Eu = features_at(V, uniq, n, boundary, taper, threads, feature)
    Eall = Eu[inv.reshape(-1)]
    Ec = Eall[: len(pts)]                                      # [count][3]
    Enb = Eall[len(pts):].reshape(len(pts), len(w), 3)
    Enb = np.where(valid[..., None], Enb, 0.0)
    S = np.abs(Ec[:, None, :] - np.asarray(w)[None, :, None] * Enb).sum(axis=1) / len(w)
    return Ec, S


# ----------------------------------------------------------------------------------------------
# Step 5: normalisation and combination (Eq. 4)
# ----------------------------------------------------------------------------------------------

def minmax_bounds(A) -> Tuple[float, float]:
    return float(np.min(A)), float(np.max(A))


def minmax(A, lo: Optional[float] = None, hi: Optional[float] = None) -> np.ndarray:
    """(A - min) / (max - min); a flat map (span <= 1e-30 max(1,|max|)) maps to 0."""
    A = _f64(A)
    if lo is None:
        lo, hi = minmax_bounds(A)
    span = hi - lo
    if span <= 1e-30 * max(1.0, abs(hi)):
        return np.zeros_like(A)
    return (A - lo) / span


def ls_weights(Shat, D, delta: float = 1e-6) -> np.ndarray:
    """W = (G + delta I)^-1 b with G = sum_p x_p x_p^T, b = sum_p x_p D_p, x_p = Shat[:, p]."""
    X = _f64(Shat).reshape(3, -1)
    d = _f64(D).reshape(-1)
    G = X @ X.T
    b = X @ d
    return np.linalg.solve(G + delta * np.eye(3), b)


def _seq_order(A) -> np.ndarray:
    """Voxel order of the sequential filters: inline sections (y) outermost, then x, then t."""
    A = np.asarray(A)
    if A.ndim == 4:
        return np.ascontiguousarray(np.transpose(A, (0, 3, 2, 1)).reshape(3, -1), dtype=np.float64)
    return np.ascontiguousarray(np.transpose(A, (2, 1, 0)).reshape(-1), dtype=np.float64)


def adapt_weights(Shat, D, method: str = "nlms", W0=(1 / 3, 1 / 3, 1 / 3), mu: float = 0.5, eps: float = 1e-8,
                  lam: float = 1.0, delta: float = 1e-6, return_trace: bool = False):
    """One sequential pass of LMS / NLMS / RLS (paper: NLMS for all results)."""
    X = _seq_order(Shat)
    d = _seq_order(D)
    N = d.size
    W = np.array(W0 if method != "rls" else (0.0, 0.0, 0.0), dtype=np.float64)
    err2 = np.empty(N, dtype=np.float64)
    L = lib()
    if method == "lms":
        rc = L.sal_oracle_lms(_dp(X), _dp(d), N, mu, _dp(W), _dp(err2))
    elif method == "nlms":
        rc = L.sal_oracle_nlms(_dp(X), _dp(d), N, mu, eps, _dp(W), _dp(err2))
    elif method == "rls":
        rc = L.sal_oracle_rls(_dp(X), _dp(d), N, lam, delta, _dp(W), _dp(err2))
    else:
        raise ValueError(method)
    _check(rc, method)
    return (W, err2) if return_trace else W


def combine(S3, weights="equal", D=None, delta: float = 1e-6, bounds=None) -> Dict[str, np.ndarray]:
    """Normalise each S_m, fit or take the weights, weighted sum, final min-max.

    weights: 'equal' | 'ls' (needs D) | 'nlms' | 'lms' | 'rls' (need D) | array of 3.
    bounds: optional frozen (lo[3], hi[3], loC, hiC) for the normalisations.
    """
    S3 = _f64(S3)
    if bounds is None:
        lo = np.array([S3[m].min() for m in range(3)])
        hi = np.array([S3[m].max() for m in range(3)])
    else:
        lo, hi = np.asarray(bounds[0], float), np.asarray(bounds[1], float)
    Shat = np.stack([minmax(S3[m], lo[m], hi[m]) for m in range(3)])
    if isinstance(weights, str):
        if weights == "equal":
            W = np.full(3, 1.0 / 3.0)
        elif weights == "ls":
            W = ls_weights(Shat, D, delta)
        else:
            W = adapt_weights(Shat, D, method=weights, delta=delta)
    else:
        W = np.asarray(weights, dtype=np.float64)
    C = np.tensordot(W, Shat, axes=1)
    if bounds is None:
        loC, hiC = minmax_bounds(C)
    else:
        loC, hiC = float(bounds[2]), float(bounds[3])
    S = minmax(C, loC, hiC)
    return {"S": S, "W": W, "Shat": Shat, "C": C, "lo": lo, "hi": hi, "loC": loC, "hiC": hiC}


def saliency(V, n: int, boundary="symmetric", taper="rect", stencil=None, weights="equal", D=None,
             delta: float = 1e-6, threads: int = 0, bounds=None, feature="abs", stride: int = 1) -> Dict[str, np.ndarray]:
    """Whole forward pass: E, raw S_m, weights and the consolidated map S."""
    if stencil is None:
        stencil = dcs_stencil()
    offsets, g, did, w = stencil
    E = features(V, n, boundary, taper, threads, feature, stride)
    S3 = center_surround(E, offsets, w, boundary, threads)
    out = combine(S3, weights, D, delta, bounds)
    out.update({"E": E, "S3": S3})
    return out


# ----------------------------------------------------------------------------------------------
# Gradient (analytic adjoint; normalisation bounds held constant)
# ----------------------------------------------------------------------------------------------

def combine_backward(fwd, W, gS):
    """Adjoint of the normalisations and Eq. 4 with the forward bounds held constant:
    returns (gS3 [3][T][X][Y], gW [3])."""
    W = np.asarray(W, dtype=np.float64)
    gS = _f64(gS)
    spanC = fwd["hiC"] - fwd["loC"]
    gC = gS / spanC if spanC > 1e-30 * max(1.0, abs(fwd["hiC"])) else np.zeros_like(gS)
    gW = np.array([np.sum(gC * fwd["Shat"][m]) for m in range(3)])
    gS3 = np.empty((3,) + gS.shape)
    for m in range(3):
        span = fwd["hi"][m] - fwd["lo"][m]
        gS3[m] = W[m] * gC / span if span > 1e-30 * max(1.0, abs(fwd["hi"][m])) else 0.0
    return gS3, gW


def center_surround_adjoint(E, gS3, offsets, w, boundary="symmetric"):
    """Adjoint of Eq. 3: returns (gE [3][T][X][Y], gw [Q]) with gw the gradient of each
    neighbour weight w_o."""
    E = _f64(E)
    gS3 = _f64(gS3)
    gE = np.empty_like(E)
    wv = _f64(w)
    gw = np.empty(len(wv), dtype=np.float64)
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    _check(lib().sal_oracle_center_surround_adjoint(_dp(E), *E.shape[1:], BOUNDARY[boundary], len(wv),
                                                    offs.ctypes.data_as(_c_int_p), _dp(wv), _dp(gS3),
                                                    _dp(gE), _dp(gw)), "center_surround_adjoint")
    return gE, gw


def direction_gradient(gw, g, did):
    """galpha_d = sum_{o in direction d} g_o gw_o  (w_o = alpha_d g_o)."""
    ndir = int(np.max(did)) + 1
    galpha = np.zeros(ndir)
    for o in range(len(gw)):
        galpha[did[o]] += gw[o] * g[o]
    return galpha


def features_adjoint(V, gE, n: int, boundary="symmetric", taper="rect", threads: int = 0,
                     feature="abs", stride: int = 1) -> np.ndarray:
    """gV = (dE/dV)^T gE through the extension (adjoint of the feature step).  stride s > 1: the
    gradient of the interpolated features goes back to the lattice (upsample_adjoint) and from there
    through the cubes of the lattice voxels.  Feature "spatial": spatial_features_adjoint (stride 1)."""
    V64 = _f64(V)
    gE = _f64(gE)
    if feature == "spatial":
        if stride != 1:
            raise ValueError("the spatial-domain reading is defined here for stride 1")
        return spatial_features_adjoint(V64, gE, n, boundary, taper)
    if stride > 1:
        gEc = upsample_adjoint(gE, stride)
        lat = np.zeros_like(gE)
        lat[:, ::stride, ::stride, ::stride] = gEc
        gE = lat
    gV = np.empty_like(V64)
    _check(lib().sal_oracle_features_adjoint(_dp(V64), *V64.shape, n, BOUNDARY[boundary], TAPER[taper],
                                             FEATURE[feature], _dp(gE), _dp(gV), threads), "features_adjoint")
    return gV


def saliency_backward(V, n: int, W, gS, boundary="symmetric", taper="rect", stencil=None, fwd=None,
                      threads: int = 0, feature="abs", stride: int = 1) -> Dict[str, np.ndarray]:
    """Gradients of sum_p gS_p S_p with respect to V, the 3 weights W and the per-direction
    alpha_d, with the min-max bounds of the forward pass held constant."""
    if stencil is None:
        stencil = dcs_stencil()
    offsets, g, did, w = stencil
    W = np.asarray(W, dtype=np.float64)
    if fwd is None:
        fwd = saliency(V, n, boundary, taper, stencil, weights=W, threads=threads, feature=feature, stride=stride)
    gS3, gW = combine_backward(fwd, W, gS)
    gE, gw = center_surround_adjoint(fwd["E"], gS3, offsets, w, boundary)
    galpha = direction_gradient(gw, g, did)
    gV = features_adjoint(V, gE, n, boundary, taper, threads, feature, stride)
    return {"gV": gV, "gW": gW, "galpha": galpha, "gE": gE, "gS3": gS3, "gw": gw}
