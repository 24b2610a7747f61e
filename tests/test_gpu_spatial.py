"""GPU parity of the spatial-domain reading of the feature step (E_m = the mean over the cube of
|IDFT(F_m)|, FP32, n in {2, 4, 8}) against the FP64 oracle, through the C ABI; the rest of the
pipeline on those features; the backward calls refuse it.  Tolerance: FP32 relative L2 <= 1e-5 per map.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RTOL = 1e-5


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
    (2, (5, 6, 9), "symmetric", "rect"),
    (4, (6, 5, 11), "periodic", "hann"),
    (4, (4, 3, 150), "zero", "rect"),      # two CTAs along y, the second ragged
    (8, (9, 10, 37), "symmetric", "rect"),
    (8, (5, 6, 20), "periodic", "hann"),
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


def test_spatial_reading_has_no_backward(sal):
    shape = (4, 4, 8)
    eng = sal.Saliency(shape, sal.Params(n=4, feature="spatial"))
    try:
        V = torch.zeros(shape, device="cuda")
        with pytest.raises(sal.SalError) as ei:
            eng.backward(V, torch.ones(3, device="cuda") / 3, torch.zeros(shape, device="cuda"))
        assert ei.value.status == 2   # SAL_ERR_UNSUPPORTED
        with pytest.raises(sal.SalError) as ei:
            sal.sal_local_spectra_project_backward(eng.h, V, torch.zeros((3,) + shape, device="cuda"),
                                                   torch.empty(shape, device="cuda"))
        assert ei.value.status == 2
    finally:
        eng.close()
