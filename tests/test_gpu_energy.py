"""GPU parity of the energy reading of the feature step (E_m = the mean over the cube's bins of
|F_m|^2 = r_m^2 |F|^2, sal_params.feature = 1) against the FP64 oracle, forward and backward, in every
precision the library builds, through the C ABI.

Tolerances as for the default feature: FP32 relative L2 <= 1e-5 per map and per gradient; the 16-bit
tensor-core forms relative L2 <= 1e-2 per map with max-abs <= 2e-2 on the normalised map S, and
relative L2 <= 1e-2 for the gradients.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _forward(sal, V, params):
    eng = sal.Saliency(V.shape, params)
    try:
        out = eng.saliency(torch.from_numpy(V).cuda(), None, intermediates=True)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        eng.close()


@pytest.mark.parametrize("n,shape,boundary,prec,tol", [
    (2, (5, 7, 40), "symmetric", "fp32", 1e-5),
    (4, (9, 6, 45), "periodic", "fp32", 1e-5),
    (8, (12, 10, 70), "zero", "fp32", 1e-5),
    (16, (8, 7, 37), "symmetric", "fp32", 1e-5),
    (32, (5, 9, 21), "symmetric", "fp32", 1e-5),
    (8, (9, 21, 37), "symmetric", "bf16", 1e-2),
    (8, (6, 16, 16), "periodic", "fp16", 1e-2),
    (16, (6, 11, 35), "symmetric", "bf16", 1e-2),
    (16, (5, 8, 16), "zero", "fp16", 1e-2),
    (32, (5, 9, 21), "symmetric", "bf16", 1e-2),
    (32, (5, 9, 21), "periodic", "fp16", 1e-2),
])
def test_energy_forward_matches_oracle(sal, n, shape, boundary, prec, tol):
    V, _ = synth.volume(synth.small_spec(shape, seed=n + shape[2], faults=2))
    p = sal.Params(n=n, boundary=boundary, prec=prec, feature="energy")
    g = _forward(sal, V, p)
    ref = oracle.saliency(V, n, boundary=boundary, stencil=oracle.dcs_stencil(p.directions, p.R, p.sigma),
                          feature="energy")
    errs = {f"E{m}": rel_l2(g["E"][m], ref["E"][m]) for m in range(3)}
    errs.update({f"S{m}": rel_l2(g["S3"][m], ref["S3"][m]) for m in range(3)})
    errs["S"] = rel_l2(g["S"], ref["S"])
    print(prec, n, shape, boundary, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= tol, (k, v)
    if prec != "fp32":
        assert np.abs(g["S"] - ref["S"]).max() <= 2e-2


@pytest.mark.parametrize("n,shape,boundary,prec,tol", [
    (2, (5, 6, 40), "symmetric", "fp32", 1e-5),
    (4, (7, 5, 37), "periodic", "fp32", 1e-5),
    (8, (10, 9, 45), "zero", "fp32", 1e-5),
    (16, (6, 5, 21), "symmetric", "fp32", 1e-5),
    (8, (7, 21, 37), "symmetric", "bf16", 1e-2),
    (8, (9, 16, 20), "zero", "fp16", 1e-2),
    (16, (6, 11, 35), "symmetric", "bf16", 1e-2),
    (16, (5, 9, 18), "periodic", "fp16", 1e-2),
])
def test_energy_spectral_adjoint_matches_oracle(sal, n, shape, boundary, prec, tol):
    V, _ = synth.volume(synth.small_spec(shape, seed=n + 3, faults=1))
    gE = synth.random_volume((3,) + shape, seed=n + 9)
    eng = sal.Saliency(shape, sal.Params(n=n, boundary=boundary, prec=prec, feature="energy"))
    try:
        gV = torch.empty(shape, dtype=torch.float32, device="cuda")
        sal.sal_local_spectra_project_backward(eng.h, _cuda(V), _cuda(gE), gV)
        torch.cuda.synchronize()
        got = gV.cpu().numpy()
    finally:
        eng.close()
    ref = oracle.features_adjoint(V, gE, n, boundary=boundary, feature="energy")
    err = rel_l2(got, ref)
    print(prec, n, shape, boundary, "gV rel-L2", f"{err:.2e}")
    assert err <= tol


@pytest.mark.parametrize("n,shape,prec,tol", [(8, (10, 12, 33), "fp32", 1e-5), (16, (6, 10, 20), "bf16", 1e-2)])
def test_energy_fused_backward(sal, n, shape, prec, tol):
    V, D = synth.volume(synth.small_spec(shape, seed=n + 1, faults=2))
    W = np.array([0.45, 0.35, 0.2])
    alpha = [1.0, 0.8, 1.2]
    params = sal.Params(n=n, alpha=alpha, prec=prec, feature="energy")
    st = oracle.dcs_stencil(params.directions, params.R, params.sigma, alpha)
    fwd = oracle.saliency(V, n, stencil=st, weights=W, feature="energy")
    gS = (fwd["S"] - D).astype(np.float32)
    ref = oracle.saliency_backward(V, n, W, gS, stencil=st, fwd=fwd, feature="energy")
    eng = sal.Saliency(shape, params)
    try:
        gV, gW, ga = eng.backward(_cuda(V), _cuda(W), _cuda(gS))
        torch.cuda.synchronize()
    finally:
        eng.close()
    errs = (rel_l2(gV.cpu().numpy(), ref["gV"]), rel_l2(gW.cpu().numpy(), ref["gW"]),
            rel_l2(ga.cpu().numpy(), ref["galpha"]))
    print(prec, n, shape, "gV gW galpha rel-L2", [f"{e:.2e}" for e in errs])
    assert max(errs) <= tol


def test_energy_feature_differs_from_default(sal):
    """The two readings are different maps (the energy weights bins quadratically)."""
    V, _ = synth.volume(synth.small_spec((6, 10, 20), seed=4, faults=1))
    a = _forward(sal, V, sal.Params(n=8))["E"]
    e = _forward(sal, V, sal.Params(n=8, feature="energy"))["E"]
    assert rel_l2(a, e) > 0.5
