"""Pins of the oracle's spatial-domain reading of the feature step (the mean over the cube of abs(f_m),
f_m the inverse DFT of the projected spectrum F_m of Eq. 1), against brute force on tiny cubes, closed
forms of plane waves, invariants, and the energy reading through Parseval."""
import numpy as np
import pytest

import oracle
import synth


def _signed(k, n):
    return k if k < n // 2 else k - n


def _brute_spatial(w):
    """From the window alone: O(n^6) DFT and inverse-DFT matrices, Eq. 1 ratios over signed indices
    (zero at DC), then the mean of abs over the cube."""
    n = w.shape[0]
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    phase = (g @ g.T) % n
    M = np.exp(-2j * np.pi * phase / n)
    F = M @ w.reshape(-1)
    s = np.array([[_signed(a, n) for a in row] for row in g], dtype=np.float64)
    r = np.sqrt((s ** 2).sum(1))
    P = np.stack([np.sqrt(s[:, 1] ** 2 + s[:, 2] ** 2), np.sqrt(s[:, 0] ** 2 + s[:, 2] ** 2),
                  np.sqrt(s[:, 0] ** 2 + s[:, 1] ** 2)])
    ratio = np.where(r > 0, P / np.where(r > 0, r, 1.0), 0.0)
    Minv = np.conj(M) / n ** 3
    return np.array([np.abs(Minv @ (F * ratio[m])).mean() for m in range(3)])


def _window(V, p, n, boundary):
    idx = [oracle.ext_index(np.arange(p[a] - n // 2, p[a] + n // 2), V.shape[a], boundary) for a in range(3)]
    return V[np.ix_(*idx)]


@pytest.mark.parametrize("n,boundary", [(2, "symmetric"), (4, "symmetric"), (4, "periodic")])
def test_spatial_reading_matches_brute_force(n, boundary):
    V = synth.random_volume((6, 5, 7), seed=n + 60)
    pts = synth.sample_points(V.shape, 5, seed=61).tolist() + [[0, 0, 0], [5, 4, 6]]
    got = oracle.spatial_features_at(V, pts, n, boundary)
    for p, e in zip(pts, got):
        ref = _brute_spatial(_window(V.astype(np.float64), p, n, boundary))
        assert np.max(np.abs(e - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


def _mean_abs_cos(n, k0):
    return np.mean(np.abs(np.cos(2 * np.pi * k0 * np.arange(n) / n)))


@pytest.mark.parametrize("n,k0", [(8, 1), (8, 3), (16, 2)])
def test_plane_wave_along_t(n, k0):
    """Only the bins (+-k0, 0, 0): P_t = 0 there, P_x / |k| = P_y / |k| = 1, so f_x = f_y = the window
    itself (zero mean) and f_t = 0."""
    T, X, Y = 2 * n, 3, 4
    t = np.arange(T)[:, None, None]
    V = np.broadcast_to(np.cos(2 * np.pi * k0 * t / n), (T, X, Y)).astype(np.float64)
    E = oracle.spatial_features_at(V, [[3, 1, 2], [n, 0, 0]], n, "periodic")
    c = _mean_abs_cos(n, k0)
    assert np.allclose(E[:, 0], 0.0, atol=1e-12)
    assert np.allclose(E[:, 1:], c, atol=1e-12)
    if n == 8 and k0 == 1:
        assert abs(c - (2 + 2 * np.sqrt(2)) / 8) <= 1e-15   # 1/8 (1 + 1 + 4 cos(pi/4))


def test_diagonal_plane_wave():
    """Bins (+-1, +-1, 0): |k| = sqrt 2, P_t = P_x = 1, P_y = sqrt 2, so E_t = E_x = c / sqrt 2, E_y = c."""
    n = 8
    t = np.arange(n)[:, None, None]
    x = np.arange(n)[None, :, None]
    V = np.broadcast_to(np.cos(2 * np.pi * (t + x) / n), (n, n, 3)).astype(np.float64)
    E = oracle.spatial_features_at(V, [[2, 5, 1]], n, "periodic")[0]
    c = _mean_abs_cos(n, 1)
    assert np.allclose(E, [c / np.sqrt(2), c / np.sqrt(2), c], atol=1e-12)


def test_constant_and_scaling():
    V = synth.random_volume((7, 6, 9), seed=62).astype(np.float64)
    pts = synth.sample_points(V.shape, 4, seed=63)
    assert np.max(oracle.spatial_features_at(np.full(V.shape, 3.5), pts, 4)) <= 1e-14 * 3.5   # FP64 rounding
    a = oracle.spatial_features_at(V, pts, 4)
    b = oracle.spatial_features_at(-2.0 * V + 7.0, pts, 4)   # a constant only moves DC
    assert np.allclose(b, 2.0 * a, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [4, 8])
def test_bounded_by_the_energy_reading(n):
    """Parseval: mean_u abs(f_m)^2 = (1/n^6) sum_k abs(F_m)^2 = E_energy / n^3, and the mean of abs is at
    most the root mean square (Cauchy-Schwarz)."""
    V, _ = synth.volume(synth.small_spec((10, 9, 11), seed=64, faults=1))
    pts = synth.sample_points(V.shape, 6, seed=65)
    Es = oracle.spatial_features_at(V, pts, n)
    Ee = oracle.features_at(V, pts, n, feature="energy")
    assert np.all(Es <= np.sqrt(Ee / n ** 3) * (1 + 1e-12))
    assert np.all(Es > 0.2 * np.sqrt(Ee / n ** 3))   # and not degenerate


@pytest.mark.parametrize("n,boundary,taper", [(4, "symmetric", "rect"), (4, "periodic", "hann"), (4, "zero", "rect"),
                                              (2, "symmetric", "rect")])
def test_spatial_adjoint_matches_exact_differences(n, boundary, taper):
    """gV[q] = d/dV[q] sum_m,p gE_m[p] E_m[p], against central differences of the forward in FP64 (no
    sample of any window's f_m crosses zero within the step: the reading is linear there up to the step's
    second order, which central differences cancel)."""
    shape = (5, 4, 6)
    V = synth.random_volume(shape, seed=70 + n).astype(np.float64)
    gE = synth.random_volume((3,) + shape, seed=71 + n).astype(np.float64)
    gV = oracle.spatial_features_adjoint(V, gE, n, boundary, taper)
    d = 1e-6
    for q in synth.sample_points(shape, 5, seed=72).tolist() + [[0, 0, 0]]:
        Vp, Vm = V.copy(), V.copy()
        Vp[tuple(q)] += d
        Vm[tuple(q)] -= d
        Lp = np.sum(gE * oracle.spatial_features(Vp, n, boundary, taper))
        Lm = np.sum(gE * oracle.spatial_features(Vm, n, boundary, taper))
        fd = (Lp - Lm) / (2 * d)
        assert abs(fd - gV[tuple(q)]) <= 1e-6 * max(1.0, abs(gV[tuple(q)])), (q, fd, gV[tuple(q)])


def test_spatial_reading_through_the_pipeline_entry_points():
    """features / features_at / center_surround_at / saliency take feature="spatial" and agree."""
    V, _ = synth.volume(synth.small_spec((6, 7, 9), seed=80, faults=1))
    E = oracle.features(V, 4, feature="spatial")
    assert np.allclose(E, oracle.spatial_features(V, 4), rtol=0, atol=0)
    pts = synth.sample_points(V.shape, 5, seed=81)
    assert np.allclose(oracle.features_at(V, pts, 4, feature="spatial"), E[:, pts[:, 0], pts[:, 1], pts[:, 2]].T)
    st = oracle.dcs_stencil()
    Ec, Sc = oracle.center_surround_at(V, pts, 4, st[0], st[3], feature="spatial")
    S3 = oracle.center_surround(E, st[0], st[3])
    assert np.allclose(Sc, S3[:, pts[:, 0], pts[:, 1], pts[:, 2]].T, rtol=1e-12, atol=1e-14)
    out = oracle.saliency(V, 4, feature="spatial")
    assert np.allclose(out["E"], E) and np.allclose(out["S3"], S3)
    with pytest.raises(ValueError):
        oracle.features(V, 4, feature="spatial", stride=2)
