"""GPU parity of the spatial-domain reading of the feature step (E_m = the mean over the cube of
|IDFT(F_m)|, FP32, n in {2, 4, 8, 16}) and of its adjoint against the FP64 oracle, through the C ABI.

Forward tolerance: FP32 relative L2 <= 1e-5 per map.  The adjoint, (1/n^3) A_m sign(f_m) per window, takes
an integer decision per sample (the sign of f_m[u]); where |f_m[u]| is within the rounding of the FP32
transforms (~1e-6 of max |f_m|) the two precisions may decide it differently, and a flipped sign moves the
gradient by 2 gE_m / n^3 times a column of A_m -- a valid subgradient of |.| at 0 in exact arithmetic, but
not the oracle's.  The parity tests therefore give gE_m = 0 to the windows whose smallest |f_m[u]| is below
2e-5 of their largest (decided by the oracle alone, with a 10x margin over the FP32 error) and compare the
rest at 1e-5; a test with every window kept bounds the effect of the undecided ones.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RTOL = 1e-5
MARGIN = 2e-5


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def sal():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_06174_gb300 as s
    s.load()
    return s


@pytest.mark.parametrize("n,shape,boundary,taper", [
    (2, (5, 6, 9), "symmetric", "rect"),      # 270 windows: 64 per CTA, the last CTA ragged
    (4, (6, 5, 11), "periodic", "hann"),
    (4, (4, 3, 150), "zero", "rect"),
    (8, (9, 10, 37), "symmetric", "rect"),
    (8, (5, 6, 20), "periodic", "hann"),
    (16, (6, 7, 40), "symmetric", "rect"),
    (16, (5, 9, 12), "periodic", "hann"),     # X, Y < n: the periodic extension wraps more than once
    (16, (3, 17, 20), "zero", "hann"),
])
def test_spatial_features_match_oracle(sal, n, shape, boundary, taper):
    V, _ = synth.volume(synth.small_spec(shape, seed=n + shape[2], faults=1))
    p = sal.Params(n=n, boundary=boundary, taper=taper, feature="spatial")
    eng = sal.Saliency(shape, p)
    try:
        out = eng.saliency(torch.from_numpy(V).cuda(), None, intermediates=True)
        torch.cuda.synchronize()
        E, S3 = out["E"].cpu().numpy(), out["S3"].cpu().numpy()
    finally:
        eng.close()
    ref = oracle.spatial_features(V, n, boundary, taper)
    errs = [rel_l2(E[m], ref[m]) for m in range(3)]
    st = oracle.dcs_stencil(p.directions, p.R, p.sigma)
    S3r = oracle.center_surround(ref, st[0], st[3], boundary=boundary)
    errs += [rel_l2(S3[m], S3r[m]) for m in range(3)]
    print(n, shape, boundary, taper, "E, S_m rel-L2", [f"{e:.1e}" for e in errs])
    assert max(errs) <= RTOL, errs


def sign_margin(V, n, boundary, taper):
    """min_u |f_m[u]| / max_u |f_m[u]| per map and voxel, [3][T][X][Y]: f_m from the oracle's projected
    spectra and numpy's inverse FFT."""
    T, X, Y = V.shape
    out = np.empty((3, T, X, Y))
    for t in range(T):
        for x in range(X):
            for y in range(Y):
                f = np.fft.ifftn(oracle.projected_spectra(V, t, x, y, n, boundary, taper), axes=(1, 2, 3)).real
                a = np.abs(f).reshape(3, -1)
                out[:, t, x, y] = a.min(axis=1) / np.maximum(a.max(axis=1), 1e-300)
    return out


def _adjoint(sal, V, gE, n, boundary, taper):
    eng = sal.Saliency(V.shape, sal.Params(n=n, boundary=boundary, taper=taper, feature="spatial"))
    try:
        gV = torch.empty(V.shape, device="cuda")
        sal.sal_local_spectra_project_backward(eng.h, torch.from_numpy(V).cuda(), torch.from_numpy(gE).cuda(), gV)
        torch.cuda.synchronize()
        return gV.cpu().numpy()
    finally:
        eng.close()


ADJ_CASES = [
    (2, (4, 11, 9), "symmetric", "rect"),     # 2 x 2 bricks of 8 x 8 windows, ragged in x and y
    (4, (5, 9, 30), "zero", "rect"),
    (8, (6, 10, 17), "periodic", "hann"),
    (8, (3, 4, 5), "symmetric", "rect"),      # the volume smaller than the window on every axis
    (16, (5, 13, 21), "symmetric", "rect"),
    (16, (4, 9, 10), "periodic", "hann"),
    (16, (9, 17, 12), "zero", "hann"),        # a Hann window's zero edge planes: many small |f|, 14 % decided
]


@pytest.mark.parametrize("n,shape,boundary,taper", ADJ_CASES)
def test_spatial_adjoint_matches_oracle(sal, n, shape, boundary, taper):
    V, _ = synth.volume(synth.small_spec(shape, seed=3 * n + shape[1], faults=1))
    rng = np.random.default_rng(n * 100 + shape[2])
    gE = rng.standard_normal((3,) + shape).astype(np.float32)
    keep = sign_margin(V, n, boundary, taper) >= MARGIN
    gE = np.where(keep, gE, 0.0).astype(np.float32)
    assert keep.sum() >= 100, keep.sum()   # enough decided (window, map) pairs to test
    ref = oracle.spatial_features_adjoint(V, gE, n, boundary, taper)
    gV = _adjoint(sal, V, gE, n, boundary, taper)
    err = rel_l2(gV, ref)
    print(n, shape, boundary, taper, f"kept {keep.mean():.3f}", f"gV rel-L2 {err:.1e}",
          f"max abs {np.max(np.abs(gV - ref)):.1e} of {np.max(np.abs(ref)):.1e}")
    assert err <= RTOL, err


@pytest.mark.parametrize("n,shape,boundary,taper", [ADJ_CASES[4], ADJ_CASES[2]])
def test_spatial_adjoint_all_windows(sal, n, shape, boundary, taper):
    """Every window kept: the undecided signs move a few voxels; relative L2 stays below 1e-3."""
    V, _ = synth.volume(synth.small_spec(shape, seed=3 * n + shape[1], faults=1))
    rng = np.random.default_rng(n * 100 + shape[2])
    gE = rng.standard_normal((3,) + shape).astype(np.float32)
    ref = oracle.spatial_features_adjoint(V, gE, n, boundary, taper)
    gV = _adjoint(sal, V, gE, n, boundary, taper)
    err = rel_l2(gV, ref)
    close = np.mean(np.abs(gV - ref) <= 1e-5 * np.max(np.abs(ref)))
    print(n, shape, boundary, taper, f"gV rel-L2 {err:.1e}", f"voxels within 1e-5 of max: {close:.4f}")
    assert err <= 1e-3, err


def test_spatial_saliency_backward_matches_oracle(sal):
    """sal_saliency_backward end to end on the spatial reading: gW and galpha depend on forward values only
    (1e-5); gV through the adjoint with every window kept (the bound of the test above)."""
    n, shape = 8, (6, 9, 20)
    V, D = synth.volume(synth.small_spec(shape, seed=5, faults=2))
    W = np.array([0.45, 0.35, 0.2])
    params = sal.Params(n=n, feature="spatial", alpha=[1.0, 0.8, 1.2])
    st = oracle.dcs_stencil(params.directions, params.R, params.sigma, [1.0, 0.8, 1.2])
    fwd = oracle.saliency(V, n, stencil=st, weights=W, feature="spatial")
    gS = (fwd["S"] - D).astype(np.float32)
    ref = oracle.saliency_backward(V, n, W, gS, stencil=st, fwd=fwd, feature="spatial")
    eng = sal.Saliency(shape, params)
    try:
        gV, gW, ga = (a.cpu().numpy() for a in eng.backward(*(torch.from_numpy(np.asarray(a, np.float32)).cuda()
                                                               for a in (V, W, gS))))
    finally:
        eng.close()
    errs = [rel_l2(gV, ref["gV"]), rel_l2(gW, ref["gW"]), rel_l2(ga, ref["galpha"])]
    print("gV, gW, galpha rel-L2", [f"{e:.1e}" for e in errs])
    assert errs[1] <= RTOL and errs[2] <= RTOL, errs
    assert errs[0] <= 1e-3, errs
