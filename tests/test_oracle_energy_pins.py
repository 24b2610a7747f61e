"""Pins of the oracle's energy feature (the squared-magnitude reading of step 3: E_m is the mean over
the cube's bins of |F_m|^2 = r_m^2 |F|^2, DC excluded) against facts fixed by mathematics:

  * Parseval with the projection identity of Eq. 1 (r_t^2 + r_x^2 + r_y^2 = 2 at every non-DC bin):
      E_t + E_x + E_y = (2/n^3) (sum_k |F|^2 - |F(0)|^2) = 2 (sum_u w^2 - (sum_u w)^2 / n^3)
    for the tapered window w around each voxel, in every border mode;
  * each E_m against numpy's FFT of the test-side window with the ratios r_m written out here;
  * a plane wave along t: only bins (+-q, 0, 0), |F| = n^3/2, so E_t = 0, E_x = E_y = n^3/2;
  * the energy is a quadratic form of V, so central differences of E are exact up to rounding:
    the oracle's adjoint against them, to 1e-9.
"""
import numpy as np
import pytest

import oracle
import synth


def _window(V, p, n, boundary, taper="rect"):
    """Test-side n^3 cube around p (offsets -n/2 .. n/2-1), extension by numpy.pad, taper applied."""
    mode = {"symmetric": "symmetric", "periodic": "wrap", "zero": "constant"}[boundary]
    P = np.pad(np.asarray(V, np.float64), n, mode=mode)
    t, x, y = (c + n - n // 2 for c in p)
    w = P[t:t + n, x:x + n, y:y + n].copy()
    if taper == "hann":
        h = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(n) / n)
        w *= h[:, None, None] * h[None, :, None] * h[None, None, :]
    return w


def _ratios_sq(n):
    """r_m(k)^2 of Eq. 1 over signed bins, [3][n][n][n], zero at DC."""
    s = np.where(np.arange(n) < n // 2, np.arange(n), np.arange(n) - n).astype(np.float64)
    i, j, k = np.meshgrid(s, s, s, indexing="ij")
    r2 = i ** 2 + j ** 2 + k ** 2
    r2[0, 0, 0] = 1.0
    out = np.stack([(j ** 2 + k ** 2) / r2, (i ** 2 + k ** 2) / r2, (i ** 2 + j ** 2) / r2])
    out[:, 0, 0, 0] = 0.0
    return out


@pytest.mark.parametrize("boundary", ["symmetric", "periodic", "zero"])
@pytest.mark.parametrize("n,taper", [(2, "rect"), (4, "rect"), (4, "hann"), (8, "rect")])
def test_energy_sum_is_twice_the_window_variance(boundary, n, taper):
    V = synth.random_volume((9, 8, 11), seed=n + len(boundary))
    E = oracle.features(V, n, boundary=boundary, taper=taper, feature="energy")
    for p in synth.sample_points(V.shape, 8, seed=n).tolist() + [[0, 0, 0], [8, 7, 10]]:
        w = _window(V, p, n, boundary, taper)
        ref = 2.0 * (np.sum(w ** 2) - np.sum(w) ** 2 / n ** 3)
        got = E[0][tuple(p)] + E[1][tuple(p)] + E[2][tuple(p)]
        assert abs(got - ref) <= 1e-12 * max(1.0, np.sum(w ** 2)), (p, got, ref)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_energy_matches_numpy_fftn(n):
    V = synth.random_volume((20, 18, 17), seed=6)
    pts = synth.sample_points(V.shape, 5, seed=n)
    E = oracle.features_at(V, pts, n, feature="energy")
    r2 = _ratios_sq(n)
    for s, p in enumerate(pts.tolist()):
        F2 = np.abs(np.fft.fftn(_window(V, p, n, "symmetric"))) ** 2
        ref = np.array([np.sum(r2[m] * F2) for m in range(3)]) / n ** 3
        assert np.allclose(E[s], ref, rtol=1e-11, atol=1e-12 * np.max(ref))


@pytest.mark.parametrize("n,q,shape", [(4, 1, (4, 4, 4)), (8, 3, (16, 8, 8))])
def test_energy_plane_wave_along_t(n, q, shape):
    t = np.arange(shape[0])[:, None, None]
    V = np.broadcast_to(np.cos(2 * np.pi * q * t / n), shape).astype(np.float64)
    E = oracle.features(V, n, boundary="periodic", feature="energy")
    assert np.max(np.abs(E[0])) <= 1e-9
    assert np.allclose(E[1], n ** 3 / 2, rtol=1e-12) and np.allclose(E[2], n ** 3 / 2, rtol=1e-12)
    # the same wave under the default feature: E_x = E_y = 1 (mean of |F_m| = 2 (n^3/2) / n^3)
    Ea = oracle.features(V, n, boundary="periodic")
    assert np.allclose(Ea[1], 1.0, atol=1e-12)


def test_energy_constant_volume_is_zero():
    V = np.full((7, 6, 9), -1.75)
    for b in ("symmetric", "periodic"):
        assert np.max(np.abs(oracle.features(V, 4, boundary=b, feature="energy"))) <= 1e-12


@pytest.mark.parametrize("boundary", ["symmetric", "periodic", "zero"])
def test_energy_adjoint_matches_exact_differences(boundary):
    n = 4
    V = synth.random_volume((7, 6, 9), seed=21).astype(np.float64)
    gE = synth.random_volume((3,) + V.shape, seed=22).astype(np.float64)
    gV = oracle.features_adjoint(V, gE, n, boundary=boundary, feature="energy")
    eps = 1e-3   # exact for a quadratic form up to rounding
    for p in synth.sample_points(V.shape, 12, seed=5).tolist() + [[0, 0, 0], [6, 5, 8]]:
        Vp = V.copy(); Vp[tuple(p)] += eps
        Vm = V.copy(); Vm[tuple(p)] -= eps
        fd = (np.sum(gE * oracle.features(Vp, n, boundary=boundary, feature="energy"))
              - np.sum(gE * oracle.features(Vm, n, boundary=boundary, feature="energy"))) / (2 * eps)
        assert abs(fd - gV[tuple(p)]) <= 1e-9 * max(1.0, abs(fd)), (p, fd, gV[tuple(p)])
