"""Pins of the oracle's 2-D section mode (the method on one section with n x n windows):

  * the section features from numpy's 2-D FFT against an O(n^4) brute-force DFT of one window;
  * a plane wave along x: only bins (+-q, 0), |F| = n^2/2, so E_x = 0 (r_x = |k| / |(j, k)| = 0 there)
    and E_y = E_0 = 1;
  * a constant section is not salient;
  * two independent codes agree: the 2-D definition against the 3-D oracle on a volume of one plane
    (symmetric or periodic extension makes every cube constant along t, so F = n F_2D at k_t = 0 and
    zero elsewhere, and r_t = 1, r_x, r_y reduce to the 2-D ratios).
"""
import numpy as np
import pytest

import oracle
import synth


def test_section_features_match_brute_force_dft():
    n = 4
    A = synth.random_volume((1, 7, 9), seed=3)[0].astype(np.float64)
    E = oracle.section_features(A, n, "zero")
    x, y = 3, 5
    P = np.pad(A, n)
    w = P[x + n - n // 2: x + n + n // 2, y + n - n // 2: y + n + n // 2]
    F = np.zeros((n, n), complex)
    for j in range(n):
        for k in range(n):
            for u in range(n):
                for v in range(n):
                    F[j, k] += w[u, v] * np.exp(-2j * np.pi * (j * u + k * v) / n)
    sb = [j if j < n // 2 else j - n for j in range(n)]
    ref = np.zeros(3)
    for j in range(n):
        for k in range(n):
            if j == 0 and k == 0:
                continue
            rad = np.hypot(sb[j], sb[k])
            ref += np.array([1.0, abs(sb[k]) / rad, abs(sb[j]) / rad]) * abs(F[j, k])
    assert np.allclose(E[:, x, y], ref / n ** 2, rtol=1e-12)


@pytest.mark.parametrize("n,q", [(4, 1), (8, 3)])
def test_section_plane_wave(n, q):
    x = np.arange(2 * n)[:, None]
    A = np.broadcast_to(np.cos(2 * np.pi * q * x / n), (2 * n, 5)).astype(np.float64)
    E = oracle.section_features(A, n, "periodic")
    assert np.max(np.abs(E[1])) <= 1e-12
    assert np.allclose(E[2], 1.0, atol=1e-12) and np.allclose(E[0], 1.0, atol=1e-12)


def test_constant_section_is_not_salient():
    out = oracle.section_saliency(np.full((9, 10), 2.5), 4, "symmetric", R=2)
    assert np.max(np.abs(out["E"])) <= 1e-12 and np.all(out["S"] == 0.0)


@pytest.mark.parametrize("n,boundary", [(4, "symmetric"), (8, "periodic"), (16, "symmetric")])
def test_section_equals_one_plane_volume(n, boundary):
    A = synth.random_volume((1, 12, 17), seed=n)[0]
    E2 = oracle.section_features(A, n, boundary)
    E3 = oracle.features(A[None], n, boundary=boundary)[:, 0]
    assert np.allclose(E2, E3, rtol=1e-12, atol=1e-12 * np.abs(E2).max())
