"""Seeded synthetic seismic volumes.

The paper evaluates on two field surveys (F3 Netherlands and Great South Basin,
Sec. 3) that are not available here.  These volumes stand in for them: layered
reflectivity convolved with a Ricker wavelet along time, deformed by folds,
planar normal faults, salt bodies and sinuous channels, plus Gaussian noise.

This module holds no arithmetic of the saliency method itself.  It is the one
input source shared by the FP64 oracle tests and the CUDA path, so that both
sides see identical volumes for a given (configuration, seed).

Layout of every array: C-contiguous [T][X][Y], float32 (T = time/depth,
X = crossline, Y = inline, as in the paper's problem statement, Sec. 2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

RICKER_F_HZ = 30.0
DT_S = 0.004
RICKER_HALF_TAPS = 12
CHUNK_X = 16  # generation proceeds in fixed X slabs, so output is chunk-invariant


@dataclasses.dataclass
class Fault:
    strike_deg: float   # angle of the strike line in the x-y plane, from +x towards +y
    dip_deg: float      # dip from horizontal, isotropic sample units
    throw: float        # hanging wall moved down by this many samples along t
    point: Tuple[float, float, float]  # (t, x, y) on the plane

    def normal(self) -> np.ndarray:
        s = math.radians(self.strike_deg)
        d = math.radians(self.dip_deg)
        # unit normal (t, x, y): horizontal part is perpendicular to the strike
        return np.array([math.cos(d), -math.sin(d) * math.sin(s), math.sin(d) * math.cos(s)])


@dataclasses.dataclass
class Salt:
    center: Tuple[float, float, float]   # (t, x, y)
    semi_axes: Tuple[float, float, float]  # (t, x, y)


@dataclasses.dataclass
class Channel:
    t_top: float
    x0: float
    amp: float
    wavelength: float
    width: float = 8.0
    thick: int = 3


@dataclasses.dataclass
class VolumeSpec:
    shape: Tuple[int, int, int]
    seed: int
    faults: List[Fault] = dataclasses.field(default_factory=list)
    salts: List[Salt] = dataclasses.field(default_factory=list)
    channels: List[Channel] = dataclasses.field(default_factory=list)
    fold_amp: float = 0.0
    fold_wavelength: float = 64.0
    noise_rel: Optional[float] = 0.1   # sigma = noise_rel * rms(signal)
    snr_db: Optional[float] = None     # used instead of noise_rel when given
    salt_fill_sigma: float = 0.3
    salt_shell_value: float = 2.0


def ricker(f_hz: float = RICKER_F_HZ, dt: float = DT_S, half: int = RICKER_HALF_TAPS) -> np.ndarray:
    tau = np.arange(-half, half + 1) * dt
    a = (math.pi * f_hz * tau) ** 2
    w = (1.0 - 2.0 * a) * np.exp(-a)
    return (w / np.abs(w).max()).astype(np.float64)


def _reflectivity_1d(rng: np.random.Generator, length: int) -> np.ndarray:
    r = np.zeros(length, dtype=np.float64)
    pos = int(rng.integers(2, 7))
    while pos < length:
        r[pos] = rng.standard_normal()
        pos += int(rng.integers(2, 7))
    return r


def _random_faults(rng, shape, count) -> List[Fault]:
    T, X, Y = shape
    out = []
    for _ in range(count):
        out.append(Fault(
            strike_deg=float(rng.uniform(0.0, 180.0)),
            dip_deg=float(rng.uniform(50.0, 80.0)),
            throw=float(rng.integers(2, 9)),
            point=(float(rng.uniform(0.2, 0.8) * T), float(rng.uniform(0.2, 0.8) * X),
                   float(rng.uniform(0.2, 0.8) * Y)),
        ))
    return out


def _random_salts(rng, shape, count) -> List[Salt]:
    T, X, Y = shape
    out = []
    for _ in range(count):
        ax = tuple(float(rng.uniform(0.08, 0.15)) * d for d in (T, X, Y))
        c = (float(rng.uniform(0.4, 0.8) * T), float(rng.uniform(0.2, 0.8) * X),
             float(rng.uniform(0.2, 0.8) * Y))
        out.append(Salt(center=c, semi_axes=ax))
    return out


def _random_channels(rng, shape, count) -> List[Channel]:
    T, X, Y = shape
    return [Channel(t_top=float(rng.uniform(0.1, 0.4) * T), x0=float(rng.uniform(0.2, 0.8) * X),
                    amp=float(rng.uniform(10, 40)), wavelength=float(rng.uniform(100, 300)))
            for _ in range(count)]


def spec_for(name: str) -> VolumeSpec:
    """Named workloads.  Sizes, structures and seeds of the five workloads."""
    if name in ("fault48", "cfg1"):
        T = X = Y = 48
        return VolumeSpec((T, X, Y), seed=0,
                          faults=[Fault(90.0, 60.0, 4.0, (T / 2, X / 2, Y / 2))], noise_rel=0.1)
    if name in ("fault128", "cfg4"):
        T = X = Y = 128
        return VolumeSpec((T, X, Y), seed=0,
                          faults=[Fault(90.0, 60.0, 4.0, (T / 2, X / 2, Y / 2))], noise_rel=0.1)
    if name in ("salt128", "cfg2"):
        shape = (128, 128, 128)
        rng = np.random.default_rng(1001)
        T, X, Y = shape
        return VolumeSpec(shape, seed=1, faults=_random_faults(rng, shape, 3),
                          salts=[Salt((0.65 * T, X / 2, Y / 2), (45.0, 30.0, 30.0))],
                          fold_amp=5.0, fold_wavelength=64.0, noise_rel=0.1)
    if name in ("precision256x384x192", "cfg3"):
        shape = (256, 384, 192)
        rng = np.random.default_rng(1002)
        return VolumeSpec(shape, seed=2, faults=_random_faults(rng, shape, 6),
                          salts=_random_salts(rng, shape, 2), fold_amp=5.0,
                          noise_rel=None, snr_db=5.0)
    if name == "section462x951":
        # a slab 8 samples thick along y; the 2-D section workload is its middle inline section (t x x)
        shape = (462, 951, 8)
        rng = np.random.default_rng(1004)
        return VolumeSpec(shape, seed=4, faults=_random_faults(rng, shape, 6),
                          salts=_random_salts(rng, shape, 1), fold_amp=5.0, noise_rel=0.1)
    if name in ("full462x951x651", "cfg5"):
        shape = (462, 951, 651)
        rng = np.random.default_rng(1003)
        return VolumeSpec(shape, seed=3, faults=_random_faults(rng, shape, 20),
                          salts=_random_salts(rng, shape, 3),
                          channels=_random_channels(rng, shape, 4), fold_amp=5.0, noise_rel=0.1)
    raise KeyError(name)


def small_spec(shape: Sequence[int], seed: int, faults: int = 1, salts: int = 0,
               fold: bool = False, noise_rel: float = 0.1) -> VolumeSpec:
    """A generator volume of arbitrary shape (used for ragged test sizes)."""
    shape = tuple(int(s) for s in shape)
    rng = np.random.default_rng(50_000 + seed)
    return VolumeSpec(shape, seed=seed, faults=_random_faults(rng, shape, faults),
                      salts=_random_salts(rng, shape, salts), fold_amp=5.0 if fold else 0.0,
                      noise_rel=noise_rel)


def _fault_offsets(spec: VolumeSpec):
    return [(f.normal(), np.asarray(f.point, dtype=np.float64), f.throw) for f in spec.faults]


def _chunk(spec: VolumeSpec, c0: int, with_mask: bool):
    """The noise-free volume (and mask) of the X slab [c0, c0 + CHUNK_X): every random draw of a slab
    comes from its own generator, so slabs can be made in any order or in parallel."""
    T, X, Y = spec.shape
    c1 = min(X, c0 + CHUNK_X)
    rng = np.random.default_rng(spec.seed)
    pad = RICKER_HALF_TAPS
    max_shift = int(math.ceil(spec.fold_amp + sum(f.throw for f in spec.faults))) + 2
    base = pad + max_shift
    r1d = _reflectivity_1d(rng, T + 2 * base + 2)
    w = ricker()
    faults = _fault_offsets(spec)
    shell_thick = [1.0 / min(s.semi_axes) for s in spec.salts]
    t_ext = np.arange(-pad, T + pad, dtype=np.float64)[:, None, None]
    y_idx = np.arange(Y, dtype=np.float64)[None, None, :]
    crng = np.random.default_rng([spec.seed, 7, c0])
    x_idx = np.arange(c0, c1, dtype=np.float64)[None, :, None]
    tau = np.broadcast_to(t_ext, (T + 2 * pad, c1 - c0, Y)).copy()
    if spec.fold_amp:
        k = 2.0 * math.pi / spec.fold_wavelength
        tau -= spec.fold_amp * np.sin(k * x_idx) * np.sin(k * y_idx)
    for nrm, p0, throw in faults:
        d = (nrm[0] * (t_ext - p0[0]) + nrm[1] * (x_idx - p0[1]) + nrm[2] * (y_idx - p0[2]))
        tau -= throw * (d > 0.0)
    # linear interpolation of the 1-D reflectivity at the deformed depth
    pos = tau + base
    i0 = np.floor(pos).astype(np.int64)
    fr = pos - i0
    R = (1.0 - fr) * r1d[i0] + fr * r1d[i0 + 1]
    for s, thick in zip(spec.salts, shell_thick):
        rho = np.sqrt(((t_ext - s.center[0]) / s.semi_axes[0]) ** 2
                      + ((x_idx - s.center[1]) / s.semi_axes[1]) ** 2
                      + ((y_idx - s.center[2]) / s.semi_axes[2]) ** 2)
        inside = rho < 1.0
        R = np.where(inside, spec.salt_fill_sigma * crng.standard_normal(R.shape), R)
        R = np.where(np.abs(rho - 1.0) <= thick, spec.salt_shell_value, R)
    for ch in spec.channels:
        xc = ch.x0 + ch.amp * np.sin(2.0 * math.pi * y_idx / ch.wavelength)
        inband = np.abs(x_idx - xc) <= ch.width / 2
        top = np.round(ch.t_top)
        R = np.where(inband & (t_ext == top), -1.5, R)
        R = np.where(inband & (t_ext > top) & (t_ext < top + ch.thick), 0.0, R)
        R = np.where(inband & (t_ext == top + ch.thick), 1.5, R)
    # convolve along t with the Ricker wavelet ('valid' part = T samples)
    out = np.zeros((T, c1 - c0, Y), dtype=np.float64)
    for k in range(2 * pad + 1):
        out += w[k] * R[k:k + T]
    clean = out.astype(np.float32)
    m = None
    if with_mask:
        tt = t_ext[pad:pad + T]
        m = np.zeros((T, c1 - c0, Y), dtype=bool)
        for nrm, p0, _ in faults:
            d = (nrm[0] * (tt - p0[0]) + nrm[1] * (x_idx - p0[1]) + nrm[2] * (y_idx - p0[2]))
            m |= np.abs(d) <= 1.0
        for s, thick in zip(spec.salts, shell_thick):
            rho = np.sqrt(((tt - s.center[0]) / s.semi_axes[0]) ** 2
                          + ((x_idx - s.center[1]) / s.semi_axes[1]) ** 2
                          + ((y_idx - s.center[2]) / s.semi_axes[2]) ** 2)
            m |= np.abs(rho - 1.0) <= thick
        m = m.astype(np.float32)
    return c0, clean, m, float(np.sum(clean.astype(np.float64) ** 2))


def make_volume(spec: VolumeSpec, with_mask: bool = True, workers: int = 0):
    """Returns (V, D): V float32 [T][X][Y]; D float32 {0,1} template mask (or None).

    D is 1 within one sample of any fault plane or on a salt shell.  workers > 1 makes the X slabs in
    that many spawned processes (the caller's main module must be safe to import, i.e. its work sits
    under `if __name__ == "__main__"`, as spawned processes import it); the result is the same bit for
    bit, since every slab has its own generators and the rms is summed in slab order.
    """
    T, X, Y = spec.shape
    clean = np.empty((T, X, Y), dtype=np.float32)
    mask = np.zeros((T, X, Y), dtype=np.float32) if with_mask else None
    starts = list(range(0, X, CHUNK_X))
    sumsq = {}
    if workers > 1 and len(starts) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            results = ex.map(_chunk, [spec] * len(starts), starts, [with_mask] * len(starts))
            for c0, cl, m, ss in results:
                clean[:, c0:c0 + cl.shape[1], :] = cl
                if with_mask:
                    mask[:, c0:c0 + cl.shape[1], :] = m
                sumsq[c0] = ss
    else:
        for c0 in starts:
            _, cl, m, ss = _chunk(spec, c0, with_mask)
            clean[:, c0:c0 + cl.shape[1], :] = cl
            if with_mask:
                mask[:, c0:c0 + cl.shape[1], :] = m
            sumsq[c0] = ss
    total = 0.0
    for c0 in starts:
        total += sumsq[c0]
    rms = math.sqrt(total / clean.size)
    if spec.snr_db is not None:
        sigma = rms * 10.0 ** (-spec.snr_db / 20.0)
    else:
        sigma = (spec.noise_rel or 0.0) * rms
    V = clean
    if sigma > 0:
        for c0 in starts:
            c1 = min(X, c0 + CHUNK_X)
            nrng = np.random.default_rng([spec.seed, 11, c0])
            V[:, c0:c1, :] += (sigma * nrng.standard_normal((T, c1 - c0, Y))).astype(np.float32)
    return V, mask


def volume(name_or_spec, with_mask: bool = True, workers: int = 0):
    spec = spec_for(name_or_spec) if isinstance(name_or_spec, str) else name_or_spec
    return make_volume(spec, with_mask=with_mask, workers=workers)


def random_volume(shape: Sequence[int], seed: int, dist: str = "normal") -> np.ndarray:
    """Plain i.i.d. random volume (for tiny edge-case tests)."""
    rng = np.random.default_rng(seed)
    if dist == "normal":
        return rng.standard_normal(tuple(shape)).astype(np.float32)
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, tuple(shape)).astype(np.float32)
    raise ValueError(dist)


def sample_points(shape: Sequence[int], count: int, seed: int) -> np.ndarray:
    """Seeded voxel coordinates [count][3] (t, x, y), int64."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, s, count) for s in shape], axis=1).astype(np.int64)
