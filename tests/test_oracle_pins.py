"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test pins the oracle to something other than itself: a brute-force O(n^6) DFT,
numpy's FFT on single windows, Parseval, the projection identity of Eq. 1, closed
forms (plane waves, constant and impulse volumes), the hand-computed worked example
in tests/golden, exact symmetries (axis permutation, integer shift) and, for the
weights, the RLS recursion against the direct least-squares solve.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import load_golden


def _window(V, p, n, boundary):
    """Test-side gather of the n^3 cube around p (offsets -n/2 .. n/2-1)."""
    T, X, Y = V.shape
    idx = []
    for a, N in zip(p, (T, X, Y)):
        ii = np.arange(a - n // 2, a + n // 2)
        if boundary == "periodic":
            ii = ii % N
        elif boundary == "symmetric":
            r = ii % (2 * N)
            ii = np.where(r < N, r, 2 * N - 1 - r)
        else:
            ii = np.where((ii >= 0) & (ii < N), ii, -1)
        idx.append(ii)
    w = np.zeros((n, n, n))
    for a in range(n):
        for b in range(n):
            for c in range(n):
                if idx[0][a] >= 0 and idx[1][b] >= 0 and idx[2][c] >= 0:
                    w[a, b, c] = V[idx[0][a], idx[1][b], idx[2][c]]
    return w


def _brute_dft(w):
    """O(n^6): F[k] = sum_u w[u] exp(-2 pi i k.u / n) as one dense n^3 x n^3 matrix."""
    n = w.shape[0]
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    phase = (g @ g.T) % n
    M = np.exp(-2j * np.pi * phase / n)
    return (M @ w.reshape(-1)).reshape(n, n, n)


@pytest.mark.parametrize("boundary", ["symmetric", "periodic", "zero"])
@pytest.mark.parametrize("n,shape", [(2, (4, 4, 4)), (4, (5, 4, 6)), (4, (8, 7, 5))])
def test_dft_matches_brute_force(boundary, n, shape):
    V = synth.random_volume(shape, seed=n + sum(shape))
    V64 = V.astype(np.float64)
    for p in synth.sample_points(shape, 6, seed=3) .tolist() + [[0, 0, 0], [s - 1 for s in shape]]:
        F = oracle.local_spectrum(V, *p, n=n, boundary=boundary)
        ref = _brute_dft(_window(V64, p, n, boundary))
        assert np.max(np.abs(F - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n", [8, 16])
def test_dft_matches_numpy_fftn(n):
    V = synth.random_volume((20, 18, 17), seed=5)
    for p in synth.sample_points(V.shape, 4, seed=n).tolist():
        F = oracle.local_spectrum(V, *p, n=n)
        ref = np.fft.fftn(_window(V.astype(np.float64), p, n, "symmetric"))
        assert np.max(np.abs(F - ref)) <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("n", [4, 8, 16])
def test_hann_taper_spectrum_matches_numpy_fftn(n):
    """The optional taper: the cube times the periodic Hann window 1/2 - 1/2 cos(2 pi u / n) on every axis,
    built here independently, then numpy's FFT."""
    V = synth.random_volume((19, 17, 21), seed=n + 40)
    h = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(n) / n)
    h3 = h[:, None, None] * h[None, :, None] * h[None, None, :]
    for p in synth.sample_points(V.shape, 4, seed=n + 41).tolist() + [[0, 0, 0]]:
        F = oracle.local_spectrum(V, *p, n=n, taper="hann")
        ref = np.fft.fftn(_window(V.astype(np.float64), p, n, "symmetric") * h3)
        assert np.max(np.abs(F - ref)) <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("n", [4, 8, 16])
def test_parseval_per_window(n):
    V, _ = synth.volume(synth.small_spec((24, 20, 22), seed=2, faults=1))
    for p in synth.sample_points(V.shape, 5, seed=11).tolist():
        F = oracle.local_spectrum(V, *p, n=n)
        w = _window(V.astype(np.float64), p, n, "symmetric")
        assert abs(np.sum(np.abs(F) ** 2) - n ** 3 * np.sum(w ** 2)) <= 1e-12 * n ** 3 * np.sum(w ** 2)


@pytest.mark.parametrize("n", [2, 4, 8])
def test_projection_identity(n):
    """Eq. 1: r_t^2 + r_x^2 + r_y^2 = 2 at every non-DC bin, so sum_m |F_m|^2 = 2 |F|^2; F_m(DC) = 0."""
    V = synth.random_volume((9, 10, 11), seed=7)
    for p in synth.sample_points(V.shape, 4, seed=n).tolist():
        F = oracle.local_spectrum(V, *p, n=n)
        Fm = oracle.projected_spectra(V, *p, n=n)
        lhs = np.sum(np.abs(Fm) ** 2, axis=0)
        rhs = 2.0 * np.abs(F) ** 2
        rhs[0, 0, 0] = 0.0
        assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(F).max() ** 2)
        assert np.all(Fm[:, 0, 0, 0] == 0)


@pytest.mark.parametrize("boundary", ["symmetric", "periodic"])
def test_constant_volume_is_not_salient(boundary):
    V = np.full((10, 9, 12), 3.25, dtype=np.float32)
    out = oracle.saliency(V, 4, boundary=boundary, stencil=oracle.dcs_stencil(R=2))
    assert np.max(np.abs(out["E"])) <= 1e-12
    assert np.max(np.abs(out["S3"])) <= 1e-12
    assert np.all(out["S"] == 0.0)


@pytest.mark.parametrize("n,q,shape", [(4, 1, (4, 4, 4)), (8, 3, (16, 8, 8)), (8, 1, (8, 5, 7))])
def test_plane_wave_along_t(n, q, shape):
    """cos(2 pi q t / n) on a periodic volume: only bins (+-q,0,0), |F| = n^3/2, so
    E_t = 0 (Eq. 1: P_t = 0 on the f_t axis) and E_x = E_y = 1 everywhere."""
    t = np.arange(shape[0])[:, None, None]
    V = np.broadcast_to(np.cos(2 * np.pi * q * t / n), shape).astype(np.float64)
    F = oracle.local_spectrum(V, 1, 2, 3, n=n, boundary="periodic")
    nz = np.argwhere(np.abs(F) > 1e-9)
    assert sorted(map(tuple, nz)) == sorted([(q, 0, 0), (n - q, 0, 0)])
    assert np.allclose(np.abs(F[q, 0, 0]), n ** 3 / 2, rtol=1e-13)
    stencil = oracle.dcs_stencil(R=2)
    out = oracle.saliency(V, n, boundary="periodic", stencil=stencil)
    E = out["E"]
    assert np.max(np.abs(E[0])) <= 1e-12
    assert np.allclose(E[1], 1.0, atol=1e-12) and np.allclose(E[2], 1.0, atol=1e-12)
    # Eq. 3 on constant E: S_m = E_m (1/Q) sum_o |1 - w_o|
    w = stencil[3]
    assert np.allclose(out["S3"][1], np.sum(np.abs(1 - w)) / len(w), atol=1e-12)


@pytest.mark.parametrize("n", [4, 8])
def test_diagonal_plane_wave_signed_bins(n):
    """cos(2 pi (t - x) / n): bins +-(1, n-1, 0), i.e. signed (1,-1,0).  With the signed
    index reading, r_t = r_x = 1/sqrt2 and r_y = 1 (unsigned indices would give
    r_t = (n-1)/sqrt(1+(n-1)^2) instead)."""
    t = np.arange(2 * n)[:, None, None]
    x = np.arange(n)[None, :, None]
    V = np.broadcast_to(np.cos(2 * np.pi * (t + (n - 1) * x) / n), (2 * n, n, 3)).astype(np.float64)
    E = oracle.features(V, n, boundary="periodic")
    assert np.allclose(E[0], 1 / math.sqrt(2), atol=1e-12)
    assert np.allclose(E[1], 1 / math.sqrt(2), atol=1e-12)
    assert np.allclose(E[2], 1.0, atol=1e-12)


def test_impulse_worked_example():
    g = load_golden("impulse_4x4x4_n2.txt")
    assert abs((3 + math.sqrt(2) + math.sqrt(2 / 3)) / 8 - g["c2"]) < 1e-7
    V = np.zeros((4, 4, 4))
    V[1, 1, 1] = 1.0
    stencil = oracle.dcs_stencil(directions=((1, 0, 0),), R=1, sigma=1.0)
    out = oracle.saliency(V, 2, boundary="periodic", stencil=stencil)
    inner = np.zeros((4, 4, 4), dtype=bool)
    inner[1:3, 1:3, 1:3] = True
    cap = np.zeros((4, 4, 4), dtype=bool)
    cap[[0, 3], 1:3, 1:3] = True
    for m in range(3):
        assert np.allclose(out["E"][m][inner], g["c2"], atol=5e-8)
        assert np.all(out["E"][m][~inner] == 0.0)
        assert np.allclose(out["S3"][m][inner], g["S_inner"], atol=5e-8)
        assert np.allclose(out["S3"][m][cap], g["S_cap"], atol=5e-8)
        assert np.all(out["S3"][m][~(inner | cap)] == 0.0)
    assert np.allclose(out["S"][inner], 1.0, atol=1e-12)
    assert np.allclose(out["S"][cap], g["S_norm_cap"], atol=5e-8)
    assert np.all(out["S"][~(inner | cap)] == 0.0)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_impulse_constant(n):
    g = load_golden("impulse_4x4x4_n2.txt")
    V = np.zeros((n + 2, n + 1, n + 3))
    V[n // 2, n // 2, n // 2] = 1.0
    E = oracle.features_at(V, [[n // 2, n // 2, n // 2]], n, boundary="zero")
    assert np.allclose(E, g[f"c{n}"], atol=5e-8)


def test_axis_permutation():
    """Swapping t and x in V and in the stencil swaps E_t and E_x (exact up to rounding)."""
    V, _ = synth.volume(synth.small_spec((14, 12, 10), seed=4, faults=1))
    st = oracle.dcs_stencil(directions=((1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 1, 1)), R=2)
    stp = (st[0][:, [1, 0, 2]], st[1], st[2], st[3])
    a = oracle.saliency(V, 4, stencil=st)
    b = oracle.saliency(np.ascontiguousarray(V.transpose(1, 0, 2)), 4, stencil=stp)
    perm = lambda A: A.transpose(1, 0, 2)
    for key in ("E", "S3"):
        assert np.allclose(b[key][0], perm(a[key][1]), rtol=1e-12, atol=1e-12)
        assert np.allclose(b[key][1], perm(a[key][0]), rtol=1e-12, atol=1e-12)
        assert np.allclose(b[key][2], perm(a[key][2]), rtol=1e-12, atol=1e-12)


def test_integer_shift_periodic():
    V = synth.random_volume((12, 10, 9), seed=9)
    st = oracle.dcs_stencil(R=2)
    a = oracle.saliency(V, 4, boundary="periodic", stencil=st)
    sh = (3, -2, 4)
    b = oracle.saliency(np.roll(V, sh, axis=(0, 1, 2)), 4, boundary="periodic", stencil=st)
    for key in ("E", "S3"):
        assert np.allclose(b[key], np.roll(a[key], sh, axis=(1, 2, 3)), rtol=1e-12, atol=1e-12)


def test_integer_shift_symmetric_interior():
    n, R = 4, 2
    big = synth.random_volume((22, 20, 21), seed=12)
    V = big[2:, 1:, 3:]
    W = big[:-2, :-1, :-3]  # W shifted by (2,1,3) relative to V
    st = oracle.dcs_stencil(R=R)
    a = oracle.saliency(V, n, stencil=st)
    b = oracle.saliency(W, n, stencil=st)
    m = n // 2 + R + 3
    sa = a["S3"][:, m:-m, m:-m, m:-m]
    sb = b["S3"][:, m + 2:V.shape[0] - m + 2, m + 1:V.shape[1] - m + 1, m + 3:V.shape[2] - m + 3]
    assert np.allclose(sa, sb, rtol=1e-12, atol=1e-12)


def test_features_at_and_center_surround_at_match_full():
    V, _ = synth.volume(synth.small_spec((11, 13, 9), seed=1, faults=1))
    st = oracle.dcs_stencil()
    E = oracle.features(V, 4)
    S3 = oracle.center_surround(E, st[0], st[3])
    pts = np.concatenate([synth.sample_points(V.shape, 20, seed=2), [[0, 0, 0], [10, 12, 8]]])
    Ec, Sc = oracle.center_surround_at(V, pts, 4, st[0], st[3])
    assert np.array_equal(Ec, E[:, pts[:, 0], pts[:, 1], pts[:, 2]].T)
    assert np.allclose(Sc, S3[:, pts[:, 0], pts[:, 1], pts[:, 2]].T, rtol=1e-14, atol=1e-15)


def test_center_surround_brute_force_loops():
    rng = np.random.default_rng(0)
    E = rng.random((3, 5, 4, 6))
    st = oracle.dcs_stencil(R=2)
    S = oracle.center_surround(E, st[0], st[3], boundary="zero")
    T, X, Y = E.shape[1:]
    ref = np.zeros_like(E)
    for m in range(3):
        for t in range(T):
            for x in range(X):
                for y in range(Y):
                    acc = 0.0
                    for o, w in zip(st[0], st[3]):
                        tt, xx, yy = t + o[0], x + o[1], y + o[2]
                        nb = E[m, tt, xx, yy] if (0 <= tt < T and 0 <= xx < X and 0 <= yy < Y) else 0.0
                        acc += abs(E[m, t, x, y] - w * nb)
                    ref[m, t, x, y] = acc / len(st[3])
    assert np.allclose(S, ref, rtol=1e-14, atol=1e-15)


def test_equal_weights_give_mean():
    rng = np.random.default_rng(1)
    S3 = rng.random((3, 6, 5, 4))
    out = oracle.combine(S3, "equal")
    Shat = np.stack([(S3[m] - S3[m].min()) / (S3[m].max() - S3[m].min()) for m in range(3)])
    mean = Shat.mean(axis=0)
    assert np.allclose(out["S"], (mean - mean.min()) / (mean.max() - mean.min()), rtol=1e-13, atol=1e-14)


def test_ls_adapts_to_single_map_and_rls_matches():
    V, D = synth.volume(synth.small_spec((16, 14, 12), seed=3, faults=2))
    out = oracle.saliency(V, 4, stencil=oracle.dcs_stencil(R=2))
    Shat = out["Shat"]
    W = oracle.ls_weights(Shat, Shat[0])
    assert np.allclose(W, [1.0, 0.0, 0.0], atol=1e-6)
    for target in (Shat[0], D):
        Wls = oracle.ls_weights(Shat, target, delta=1e-6)
        Wrls = oracle.adapt_weights(Shat, target, "rls", lam=1.0, delta=1e-6)
        assert np.allclose(Wrls, Wls, rtol=1e-9, atol=1e-10)


def test_adaptive_filters_converge_rls_fastest():
    """The LMS family all reduce the a-priori error; RLS reaches a given MSE first."""
    V, _ = synth.volume(synth.small_spec((20, 18, 16), seed=6, faults=2))
    out = oracle.saliency(V, 4, stencil=oracle.dcs_stencil(R=2))
    Shat = out["Shat"]
    target = Shat[0]
    traces = {}
    for m in ("lms", "nlms", "rls"):
        W, e2 = oracle.adapt_weights(Shat, target, m, mu=0.05 if m == "lms" else 0.5, return_trace=True)
        traces[m] = np.convolve(e2, np.ones(200) / 200, mode="valid")
        assert traces[m][-1] < traces[m][0]
    thr = 0.01 * traces["nlms"][0]
    first = {m: int(np.argmax(tr < thr)) if np.any(tr < thr) else len(tr) for m, tr in traces.items()}
    assert first["rls"] <= first["nlms"]


def _away_from_fd_kinks(V, n, boundary, candidates, count, eps):
    """Entries every containing window of which has no non-DC bin with ZERO_BIN L1 < |F| <= 100 eps.

    A central difference of step eps moves F by at most 8 eps (a voxel enters a cube at most 8 times
    through the symmetric extension, each time with a unit twiddle), so below 100 eps it can cross
    the kink of |F| at F = 0 and is no check of the derivative there.  Bins at or below the FP64
    zero band (exact zeros of the extension) stay zero under any perturbation of the volume: the
    extension keeps their symmetry, so the difference and the zero subgradient both give 0."""
    keep = []
    for q in candidates:
        ok = True
        for ut in range(n):
            for ux in range(n):
                for uy in range(n):
                    p = [int(q[0]) + n // 2 - ut, int(q[1]) + n // 2 - ux, int(q[2]) + n // 2 - uy]
                    if not all(0 <= p[a] < V.shape[a] for a in range(3)):
                        continue
                    F = oracle.local_spectrum(V, *p, n=n, boundary=boundary)
                    l1 = np.abs(_window(V, p, n, boundary)).sum()
                    m = np.abs(F).ravel()[1:]
                    if np.any((m > oracle.ZERO_BIN * l1) & (m <= 100 * eps)):
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            keep.append(q)
        if len(keep) == count:
            break
    assert len(keep) == count
    return np.array(keep)


def _frozen_objective(V, n, W, gS, st, fwd, boundary):
    out = oracle.saliency(V, n, boundary=boundary, stencil=st, weights=W,
                          bounds=(fwd["lo"], fwd["hi"], fwd["loC"], fwd["hiC"]))
    return float(np.sum(gS * out["S"]))


@pytest.mark.parametrize("boundary", ["symmetric", "zero"])
def test_gradient_matches_finite_differences(boundary):
    """Central differences on the FP64 oracle with the min-max bounds frozen.

    eps = 1e-6: the map is only piecewise smooth (|.| in Eq. 3 and |F| at 0), and on a
    small noisy volume a step of 1e-3 crosses kinks of the center-surround terms."""
    n = 4
    V, D = synth.volume(synth.small_spec((10, 9, 11), seed=8, faults=1))
    V = V.astype(np.float64)
    st = oracle.dcs_stencil(R=2, alpha=[1.0, 0.8, 1.2])
    W = np.array([0.5, 0.3, 0.2])
    fwd = oracle.saliency(V, n, boundary=boundary, stencil=st, weights=W)
    gS = fwd["S"] - D
    bw = oracle.saliency_backward(V, n, W, gS, boundary=boundary, stencil=st, fwd=fwd)
    eps = 1e-6
    idx = _away_from_fd_kinks(V, n, boundary, synth.sample_points(V.shape, 64, seed=1234), 16, eps)
    fd = []
    for p in idx:
        Vp = V.copy(); Vp[tuple(p)] += eps
        Vm = V.copy(); Vm[tuple(p)] -= eps
        fd.append((_frozen_objective(Vp, n, W, gS, st, fwd, boundary)
                   - _frozen_objective(Vm, n, W, gS, st, fwd, boundary)) / (2 * eps))
    fd = np.array(fd)
    an = bw["gV"][idx[:, 0], idx[:, 1], idx[:, 2]]
    assert np.linalg.norm(fd - an) <= 1e-5 * np.linalg.norm(an)
    # combination weights
    fdw = []
    for m in range(3):
        Wp = W.copy(); Wp[m] += eps
        Wm = W.copy(); Wm[m] -= eps
        fdw.append((_frozen_objective(V, n, Wp, gS, st, fwd, boundary)
                    - _frozen_objective(V, n, Wm, gS, st, fwd, boundary)) / (2 * eps))
    assert np.allclose(fdw, bw["gW"], rtol=1e-6, atol=1e-9)
    # per-direction alpha
    fda = []
    alpha = np.array([1.0, 0.8, 1.2])
    for d in range(3):
        ap = alpha.copy(); ap[d] += eps
        am = alpha.copy(); am[d] -= eps
        stp = oracle.dcs_stencil(R=2, alpha=ap)
        stm = oracle.dcs_stencil(R=2, alpha=am)
        fda.append((_frozen_objective(V, n, W, gS, stp, fwd, boundary)
                    - _frozen_objective(V, n, W, gS, stm, fwd, boundary)) / (2 * eps))
    assert np.allclose(fda, bw["galpha"], rtol=1e-5, atol=1e-8)


def test_feature_adjoint_at_small_bins_matches_finite_differences():
    """The adjoint of step 3 at cubes holding bins of tiny but non-zero magnitude (2^-40 < |F| / L1 <=
    2^-19, the band an adjoint tuned to FP32 rounding would zero): central differences of
    L = sum gE . E with a step small enough (1e-7) not to cross the kink of any of those bins.  A zero
    subgradient on real bins fails here; the exact zeros of the symmetric extension (|F| / L1 below
    2^-40, unchanged by any perturbation) take the zero subgradient on both sides."""
    n, shape = 8, (9, 7, 33)
    V, _ = synth.volume(synth.small_spec(shape, seed=n + 100, faults=1))
    V = V.astype(np.float64)
    gE = synth.random_volume((3,) + shape, seed=15).astype(np.float64)
    small = oracle.band_count(V, n, "symmetric", lo=oracle.ZERO_BIN, hi=2.0 ** -19) > 0
    assert small.sum() >= 5                     # the input does hold such cubes
    foot = oracle.adjoint_footprint(small, n, "symmetric")
    eps = 1e-7
    rng = np.random.default_rng(5)
    cand = np.argwhere(foot)
    cand = cand[rng.permutation(len(cand))]
    idx = _away_from_fd_kinks(V, n, "symmetric", cand, 12, eps)
    gV = oracle.features_adjoint(V, gE, n, boundary="symmetric")

    fd = []
    for p in idx:
        Vp = V.copy(); Vp[tuple(p)] += eps
        Vm = V.copy(); Vm[tuple(p)] -= eps
        # cubes that do not contain p give bit-identical features on both sides: the difference is
        # formed per voxel before the sum, so only the changed cubes contribute rounding
        dE = oracle.features(Vp, n, boundary="symmetric") - oracle.features(Vm, n, boundary="symmetric")
        fd.append(float(np.sum(gE * dE)) / (2 * eps))
    fd = np.array(fd)
    an = gV[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an), (fd, an)


def _two_samples():
    # [3][T=1][X=1][Y=2]: the filters visit y outermost, so sample 1 is y = 0, sample 2 is y = 1
    S = np.zeros((3, 1, 1, 2))
    S[:, 0, 0, 0] = (1.0, 0.0, 0.5)
    S[:, 0, 0, 1] = (0.0, 1.0, 1.0)
    D = np.array([[[1.0, 0.0]]])
    return S, D


@pytest.mark.parametrize("method", ["lms", "nlms"])
def test_adaptive_filters_two_step_golden(method):
    """LMS and NLMS against the hand-derived two-sample runs in tests/golden (exact fractions)."""
    gold = load_golden("adaptive_two_step.txt")
    S, D = _two_samples()
    W, err2 = oracle.adapt_weights(S, D, method=method, mu=0.5, eps=0.0, return_trace=True)
    assert np.allclose(W, [gold[f"{method}_W_t"], gold[f"{method}_W_x"], gold[f"{method}_W_y"]], rtol=0, atol=1e-15)
    assert np.allclose(err2, [gold[f"{method}_e1sq"], gold[f"{method}_e2sq"]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("mu,eps", [(1.0, 0.0), (0.5, 0.0), (0.3, 0.25)])
def test_nlms_a_posteriori_error(mu, eps):
    """One NLMS step scales the error of its own sample by exactly 1 - mu |x|^2 / (eps + |x|^2): with
    mu = 1, eps = 0 the updated weights reproduce the sample (d - W_new . x = 0) for any x != 0.  A
    missing or misplaced normaliser, or mu applied twice, breaks this identity."""
    rng = np.random.default_rng(11)
    W = np.array([1 / 3, 1 / 3, 1 / 3])
    for _ in range(20):
        x = rng.uniform(0.05, 1.0, 3)
        d = rng.uniform(0.0, 1.0)
        S = x.reshape(3, 1, 1, 1)
        e = d - W @ x
        W_new = oracle.adapt_weights(S, np.array([[[d]]]), method="nlms", W0=W, mu=mu, eps=eps)
        nx = x @ x
        assert abs((d - W_new @ x) - e * (1.0 - mu * nx / (eps + nx))) <= 1e-14
        W = W_new


def test_lms_step_is_the_gradient_step():
    """One LMS step is a step of mu/2 down the gradient of the squared error e^2 = (d - W.x)^2 (whose
    gradient is -2 e x), checked by central differences of e^2 itself."""
    rng = np.random.default_rng(12)
    W = rng.uniform(-1, 1, 3)
    x = rng.uniform(0, 1, 3)
    d = 0.7
    mu = 0.25
    W_new = oracle.adapt_weights(x.reshape(3, 1, 1, 1), np.array([[[d]]]), method="lms", W0=W, mu=mu)
    h = 1e-6
    grad = np.array([((d - (W + h * np.eye(3)[m]) @ x) ** 2 - (d - (W - h * np.eye(3)[m]) @ x) ** 2) / (2 * h)
                     for m in range(3)])
    assert np.allclose(W_new, W - 0.5 * mu * grad, rtol=0, atol=1e-9)
