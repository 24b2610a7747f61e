"""The seeded synthetic seismic volumes that stand in for the paper's field surveys: the recipe's
properties (wavelet, layering, fault throw, noise level, template mask), determinism and the
slab-by-slab generation (no GPU)."""
import math

import numpy as np
import pytest

import synth
from synth.seismic import Fault, VolumeSpec, make_volume, ricker


def test_ricker_wavelet_shape():
    """30 Hz at 4 ms, 25 taps, peak 1 at zero lag, symmetric; zero crossings at +-1/(pi f sqrt 2) = 7.5 ms
    (between taps 1 and 2), deepest side lobes at +-sqrt(3/2)/(pi f) = 13 ms (tap 3)."""
    w = ricker()
    assert w.shape == (25,) and w[12] == 1.0 and np.allclose(w, w[::-1])
    assert w[13] > 0 > w[14]
    assert np.argmin(w[12:]) == 3
    assert abs(1.0 / (math.pi * 30.0 * math.sqrt(2.0)) - 0.0075) < 1e-4


def _plain(shape, **kw):
    return VolumeSpec(tuple(shape), seed=kw.pop("seed", 5), noise_rel=kw.pop("noise_rel", None), **kw)


def test_undeformed_traces_are_identical():
    V, _ = make_volume(_plain((40, 6, 7)), with_mask=False)
    assert np.all(V == V[:, :1, :1])
    assert np.std(V) > 0.1


def test_normal_fault_moves_the_hanging_wall_down_by_its_throw():
    """A vertical fault striking along y through x = 10: on the side the normal points to (x < 10) the
    reflectivity is read `throw` samples shallower, so those traces are the others delayed by the throw."""
    T, X, Y, throw = 60, 20, 5, 4
    V, D = make_volume(_plain((T, X, Y), faults=[Fault(90.0, 90.0, float(throw), (T / 2, 10.0, 2.0))]))
    near, far = V[:, 3, 2], V[:, 15, 2]
    assert np.allclose(near[throw + 13:T - 13], far[13:T - 13 - throw], atol=1e-6)
    assert not np.allclose(near, far)
    # template mask: 1 within one sample of the plane x = 10 (x = 9 and 11 sit on the band's edge), 0 beyond
    assert np.all(D[:, 10, :] == 1.0) and np.all(D[:, :8, :] == 0.0) and np.all(D[:, 13:, :] == 0.0)


@pytest.mark.parametrize("noise_rel,snr_db,expect", [(0.1, None, 0.1), (None, 5.0, 10 ** (-5.0 / 20))])
def test_noise_level(noise_rel, snr_db, expect):
    shape = (48, 32, 40)
    clean, _ = make_volume(_plain(shape, faults=[Fault(30.0, 60.0, 3.0, (24.0, 16.0, 20.0))]), with_mask=False)
    noisy, _ = make_volume(VolumeSpec(shape, seed=5, faults=[Fault(30.0, 60.0, 3.0, (24.0, 16.0, 20.0))],
                                      noise_rel=noise_rel, snr_db=snr_db), with_mask=False)
    rel = np.sqrt(np.mean((noisy.astype(np.float64) - clean) ** 2)) / np.sqrt(np.mean(clean.astype(np.float64) ** 2))
    assert abs(rel - expect) <= 0.02 * expect


def test_generation_is_slab_invariant():
    """Volumes are generated in slabs of 16 x-columns, each slab from its own seeded stream: a wider
    volume with the same spec repeats the narrower one's first slabs exactly (noise off: its level
    depends on the whole volume's rms)."""
    f = [Fault(40.0, 70.0, 3.0, (20.0, 8.0, 9.0))]
    a, _ = make_volume(_plain((30, 20, 18), faults=f), with_mask=False)
    b, _ = make_volume(_plain((30, 40, 18), faults=f), with_mask=False)
    assert np.array_equal(a[:, :16], b[:, :16])


def test_named_workloads_are_deterministic():
    a, da = synth.volume("fault48")
    b, db = synth.volume("fault48")
    assert a.shape == (48, 48, 48) and a.dtype == np.float32
    assert np.array_equal(a, b) and np.array_equal(da, db)
    assert 0.0 < da.mean() < 0.2   # the mask marks a thin band around the fault plane
    c, _ = synth.volume(synth.small_spec((12, 11, 13), seed=1))
    d, _ = synth.volume(synth.small_spec((12, 11, 13), seed=2))
    assert not np.array_equal(c, d)


def test_sample_points_in_bounds_and_seeded():
    p = synth.sample_points((5, 7, 9), 200, seed=3)
    assert p.shape == (200, 3) and p.dtype == np.int64
    assert np.all(p >= 0) and np.all(p < np.array([5, 7, 9]))
    assert np.array_equal(p, synth.sample_points((5, 7, 9), 200, seed=3))
