"""Host checks of the two identities the FP32 adjoint's sliding y-passes rest on (no GPU; plain numpy, FP64).

For one (k_t, k_x) row, G2 sampled along y, and a run of r <= n outputs starting at y_r:
1. the forward stage 3 with the phase anchored at the run's start, Ft_j[k] = F_{y_r + j}[k] w^(k j)
   (w = e^(-2 pi i / n)), follows Ft_{j+1} = Ft_j + (G2[y_r + j + n] - G2[y_r + j]) w^(k j), and |Ft| = |F|;
2. the inverse DFT along y of the run, dG2[y_r + p] = sum over the outputs j with j <= p < j + n of
   sum_k Gamma_j[k] e^(2 pi i k (p - j) / n), equals the single-point inverse DFT z(P, p) =
   sum_k P[k] e^(2 pi i k p / n) of prefix sums P_i of Gamma~_j = Gamma_j w^(k j):
   z(P_p, p) for p < r - 1, z(P_{r-1}, p) for r - 1 <= p < n, z(P_{r-1}, i) - z(P_i, i) at p = n + i.
"""
import numpy as np
import pytest


def _forward_direct(G2, n, r):
    k = np.arange(n)
    return np.array([[np.sum(G2[j:j + n] * np.exp(-2j * np.pi * kk * np.arange(n) / n)) for kk in k]
                     for j in range(r)])


@pytest.mark.parametrize("n,r", [(8, 4), (16, 8), (16, 16), (4, 2), (16, 1)])
def test_anchored_forward_recursion(n, r):
    rng = np.random.default_rng(n * 7 + r)
    G2 = rng.standard_normal(r + n - 1) + 1j * rng.standard_normal(r + n - 1)
    F = _forward_direct(G2, n, r)
    k = np.arange(n)
    Ft = np.empty_like(F)
    Ft[0] = F[0]
    for j in range(r - 1):
        Ft[j + 1] = Ft[j] + (G2[j + n] - G2[j]) * np.exp(-2j * np.pi * k * j / n)
    anchored = F * np.exp(-2j * np.pi * np.outer(np.arange(r), k) / n)
    assert np.max(np.abs(Ft - anchored)) <= 1e-12 * np.max(np.abs(F))
    assert np.allclose(np.abs(Ft), np.abs(F), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n,r", [(8, 4), (16, 8), (16, 16), (4, 2), (16, 1)])
def test_inverse_by_prefix_sums(n, r):
    rng = np.random.default_rng(n * 11 + r)
    Gam = rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n))
    k = np.arange(n)
    direct = np.zeros(r + n - 1, complex)
    for j in range(r):
        for u in range(n):
            direct[j + u] += np.sum(Gam[j] * np.exp(2j * np.pi * k * u / n))
    Gt = Gam * np.exp(-2j * np.pi * np.outer(np.arange(r), k) / n)
    P = np.cumsum(Gt, axis=0)

    def z(Pi, p):
        return np.sum(Pi * np.exp(2j * np.pi * k * p / n))

    slid = np.zeros_like(direct)
    for p in range(r - 1):
        slid[p] = z(P[p], p)
        slid[n + p] = z(P[r - 1], p) - z(P[p], p)
    for p in range(r - 1, n):
        slid[p] = z(P[r - 1], p)
    assert np.max(np.abs(slid - direct)) <= 1e-12 * np.max(np.abs(direct))


def test_prefix_form_point_evaluations():
    """r - 1 + n point evaluations per run replace r n (the work the sliding inverse saves)."""
    for n, r in ((8, 4), (16, 8)):
        assert (r - 1) + n < r * n
