"""GPU parity of the stride-s windows (cubes only at voxels whose indices are multiples of s, windows
overlapping by n - s of n, more than half for s < n/2; the features interpolated trilinearly in
between) against the FP64 oracle, through the C ABI, in every precision, forward and backward.

Tolerances as for stride 1: FP32 relative L2 <= 1e-5 per map; the 16-bit tensor-core forms relative
L2 <= 1e-2 per map and max-abs <= 2e-2 on the normalised map S.  Volumes are not multiples of s, so
the held values past the last lattice point are covered.
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


@pytest.mark.parametrize("n,s,shape,boundary,prec,feature,tol", [
    (8, 2, (11, 9, 37), "symmetric", "fp32", "abs", 1e-5),
    (8, 3, (10, 8, 35), "periodic", "fp32", "energy", 1e-5),
    (16, 4, (9, 10, 21), "zero", "fp32", "abs", 1e-5),
    (32, 5, (7, 9, 21), "symmetric", "fp32", "abs", 1e-5),
    (8, 2, (9, 21, 37), "symmetric", "bf16", "abs", 1e-2),
    (16, 3, (8, 11, 35), "symmetric", "fp16", "abs", 1e-2),
    (16, 2, (7, 10, 20), "periodic", "bf16", "energy", 1e-2),
    (32, 4, (7, 9, 21), "symmetric", "bf16", "abs", 1e-2),
])
def test_stride_forward_matches_oracle(sal, n, s, shape, boundary, prec, feature, tol):
    V, _ = synth.volume(synth.small_spec(shape, seed=n + s + shape[2], faults=2))
    p = sal.Params(n=n, boundary=boundary, prec=prec, feature=feature, stride=s)
    eng = sal.Saliency(shape, p)
    try:
        out = eng.saliency(torch.from_numpy(V).cuda(), None, intermediates=True)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        eng.close()
    ref = oracle.saliency(V, n, boundary=boundary, stencil=oracle.dcs_stencil(p.directions, p.R, p.sigma),
                          feature=feature, stride=s)
    errs = {f"E{m}": rel_l2(g["E"][m], ref["E"][m]) for m in range(3)}
    errs.update({f"S{m}": rel_l2(g["S3"][m], ref["S3"][m]) for m in range(3)})
    errs["S"] = rel_l2(g["S"], ref["S"])
    print(prec, n, s, shape, boundary, feature, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= tol, (k, v)
    if prec != "fp32":
        assert np.abs(g["S"] - ref["S"]).max() <= 2e-2


@pytest.mark.parametrize("taper", ["hann", "rect"])
def test_stride_lattice_matches_stride_one(sal, taper):
    """On the lattice the stride-3 features are the per-voxel features (FP32).  With the Hann taper both
    runs take the direct stage-3 sum, so they agree bit for bit (the interpolation is exact there:
    weights 0 and 1); with the rect cube stride 1 takes the sliding recursion along y, within 1e-6."""
    shape = (10, 9, 40)
    V, _ = synth.volume(synth.small_spec(shape, seed=3, faults=1))
    Es = []
    for s in (1, 3):
        eng = sal.Saliency(shape, sal.Params(n=8, stride=s, taper=taper))
        try:
            out = eng.saliency(torch.from_numpy(V).cuda(), None, intermediates=True)
            torch.cuda.synchronize()
            Es.append(out["E"].cpu().numpy())
        finally:
            eng.close()
    lat = np.ix_(range(3), range(0, 10, 3), range(0, 9, 3), range(0, 40, 3))
    if taper == "hann":
        assert np.array_equal(Es[0][lat], Es[1][lat])
    else:
        assert rel_l2(Es[0][lat], Es[1][lat]) <= 1e-6


def test_stride_arguments(sal):
    for n, s in ((8, 4), (4, 2), (16, 0)):   # s must be 1 or 1 < s < n/2
        with pytest.raises(sal.SalError):
            sal.Saliency((8, 8, 8), sal.Params(n=n, stride=s))


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("n,s,shape,boundary,prec,feature,tol", [
    (8, 2, (9, 7, 37), "symmetric", "fp32", "abs", 1e-5),
    (8, 3, (10, 8, 35), "periodic", "fp32", "energy", 1e-5),
    (16, 4, (9, 6, 21), "zero", "fp32", "abs", 1e-5),
    (8, 2, (9, 21, 37), "symmetric", "bf16", "abs", 1e-2),
    (16, 3, (8, 11, 35), "symmetric", "fp16", "energy", 1e-2),
])
def test_stride_spectral_adjoint_matches_oracle(sal, n, s, shape, boundary, prec, feature, tol):
    V, _ = synth.volume(synth.small_spec(shape, seed=n + 3 * s, faults=1))
    gE = synth.random_volume((3,) + shape, seed=n + s)
    eng = sal.Saliency(shape, sal.Params(n=n, boundary=boundary, prec=prec, feature=feature, stride=s))
    try:
        gV = torch.empty(shape, dtype=torch.float32, device="cuda")
        sal.sal_local_spectra_project_backward(eng.h, _cuda(V), _cuda(gE), gV)
        torch.cuda.synchronize()
        got = gV.cpu().numpy()
    finally:
        eng.close()
    ref = oracle.features_adjoint(V, gE, n, boundary=boundary, feature=feature, stride=s)
    err = rel_l2(got, ref)
    print(prec, n, s, shape, boundary, feature, "gV rel-L2", f"{err:.2e}")
    assert err <= tol


def test_stride_spectral_adjoint_in_slabs(sal):
    """A budget that leaves room for one lattice plane of bricks at a time."""
    n, s, shape = 8, 2, (11, 9, 40)
    V, _ = synth.volume(synth.small_spec(shape, seed=9, faults=1))
    gE = synth.random_volume((3,) + shape, seed=10)
    base = sal.Saliency(shape, sal.Params(n=n, stride=s))
    created = sal.sal_workspace_size(base.h)
    base.close()
    N = int(np.prod(shape))
    nseg = -(-shape[2] // 32)
    per_t = shape[1] * nseg * n * n * (32 + n - 1) * 4
    per_ext = per_t // n
    budget = created + 2 * 3 * N * 4 + 1216 * 64 * 8 + per_t + (n - s) * per_ext + s * per_ext
    eng = sal.Saliency(shape, sal.Params(n=n, stride=s, hbm_budget_bytes=budget))
    try:
        gV = torch.empty(shape, dtype=torch.float32, device="cuda")
        sal.sal_local_spectra_project_backward(eng.h, _cuda(V), _cuda(gE), gV)
        torch.cuda.synchronize()
        got = gV.cpu().numpy()
    finally:
        eng.close()
    ref = oracle.features_adjoint(V, gE, n, stride=s)
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)


@pytest.mark.parametrize("n,s,shape,prec,tol", [(8, 2, (10, 12, 33), "fp32", 1e-5), (16, 3, (7, 10, 20), "bf16", 1e-2)])
def test_stride_fused_backward(sal, n, s, shape, prec, tol):
    V, D = synth.volume(synth.small_spec(shape, seed=n + s, faults=2))
    W = np.array([0.45, 0.35, 0.2])
    alpha = [1.0, 0.8, 1.2]
    params = sal.Params(n=n, alpha=alpha, prec=prec, stride=s)
    st = oracle.dcs_stencil(params.directions, params.R, params.sigma, alpha)
    fwd = oracle.saliency(V, n, stencil=st, weights=W, stride=s)
    gS = (fwd["S"] - D).astype(np.float32)
    ref = oracle.saliency_backward(V, n, W, gS, stencil=st, fwd=fwd, stride=s)
    eng = sal.Saliency(shape, params)
    try:
        gV, gW, ga = eng.backward(_cuda(V), _cuda(W), _cuda(gS))
        torch.cuda.synchronize()
    finally:
        eng.close()
    errs = (rel_l2(gV.cpu().numpy(), ref["gV"]), rel_l2(gW.cpu().numpy(), ref["gW"]),
            rel_l2(ga.cpu().numpy(), ref["galpha"]))
    print(prec, n, s, shape, "gV gW galpha rel-L2", [f"{e:.2e}" for e in errs])
    assert max(errs) <= tol
