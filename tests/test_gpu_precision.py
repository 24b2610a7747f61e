"""Precision form: the local-DFT contraction on the tensor cores in BF16 / FP16 with FP32
accumulation, against the FP64 oracle.

Tolerance of the 16-bit forms: relative L2 <= 1e-2 per map and max-abs <= 2e-2 on the normalised
[0, 1] map S.
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


def _run(sal, V, params, D=None):
    eng = sal.Saliency(V.shape, params)
    try:
        out = eng.saliency(torch.from_numpy(V).cuda(), None if D is None else torch.from_numpy(D).cuda(),
                           intermediates=True)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        eng.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,shape,boundary", [
    (8, (9, 21, 37), "symmetric"),
    (8, (6, 16, 16), "periodic"),
    (16, (6, 11, 35), "symmetric"),
    (16, (5, 8, 16), "zero"),
])
def test_tensor_core_forward_matches_oracle(sal, prec, n, shape, boundary):
    V, _ = synth.volume(synth.small_spec(shape, seed=n + shape[1], faults=2))
    p = sal.Params(n=n, boundary=boundary, prec=prec)
    g = _run(sal, V, p)
    ref = oracle.saliency(V, n, boundary=boundary,
                          stencil=oracle.dcs_stencil(p.directions, p.R, p.sigma))
    errs = {f"E{m}": rel_l2(g["E"][m], ref["E"][m]) for m in range(3)}
    errs.update({f"S{m}": rel_l2(g["S3"][m], ref["S3"][m]) for m in range(3)})
    errs["S"] = rel_l2(g["S"], ref["S"])
    print(prec, n, shape, {k: f"{v:.2e}" for k, v in errs.items()}, "maxabs", np.abs(g["S"] - ref["S"]).max())
    for k, v in errs.items():
        assert v <= 1e-2, (k, v)
    assert np.abs(g["S"] - ref["S"]).max() <= 2e-2


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tensor_core_salt128_n16_sampled(sal, prec):
    """The 128^3 workload: raw maps at seeded voxels against the oracle, and the normalised map
    against the FP32 GPU form."""
    V, _ = synth.volume("salt128")
    g = _run(sal, V, sal.Params(n=16, prec=prec))
    g32 = _run(sal, V, sal.Params(n=16, prec="fp32"))
    p = sal.Params(n=16)
    st = oracle.dcs_stencil(p.directions, p.R, p.sigma)
    pts = synth.sample_points(V.shape, 40, seed=5)
    Ec, Sc = oracle.center_surround_at(V, pts, 16, st[0], st[3])
    for m in range(3):
        assert rel_l2(g["E"][m][pts[:, 0], pts[:, 1], pts[:, 2]], Ec[:, m]) <= 1e-2
        assert rel_l2(g["S3"][m][pts[:, 0], pts[:, 1], pts[:, 2]], Sc[:, m]) <= 1e-2
    assert rel_l2(g["S"], g32["S"]) <= 1e-2
    assert np.abs(g["S"] - g32["S"]).max() <= 2e-2


@pytest.mark.parametrize("n,precs", [(8, ("bf16", "fp16")), (16, ("bf16", "fp16")), (32, ("bf16",))])
def test_precision_workload_256x384x192_sampled(sal, n, precs):
    """The precision-form workload at full size (6 faults, 2 salt bodies, SNR 5 dB): raw E_m and S_m of
    the tensor-core forms at seeded voxels against the FP64 oracle, and the normalised map against the
    FP32 GPU form (the global min-max couples every voxel, so S is compared whole to FP32)."""
    V, _ = synth.volume("precision256x384x192")
    p = sal.Params(n=n)
    st = oracle.dcs_stencil(p.directions, p.R, p.sigma)
    pts = synth.sample_points(V.shape, 24 if n < 32 else 8, seed=7)
    Ec, Sc = oracle.center_surround_at(V, pts, n, st[0], st[3])
    g32 = _run(sal, V, sal.Params(n=n, prec="fp32"))
    for prec in precs:
        g = _run(sal, V, sal.Params(n=n, prec=prec))
        errs = [rel_l2(g["E"][m][pts[:, 0], pts[:, 1], pts[:, 2]], Ec[:, m]) for m in range(3)]
        errs += [rel_l2(g["S3"][m][pts[:, 0], pts[:, 1], pts[:, 2]], Sc[:, m]) for m in range(3)]
        print(prec, n, "E/S_m sampled rel-L2", [f"{e:.2e}" for e in errs], "S vs FP32",
              f"{rel_l2(g['S'], g32['S']):.2e}", f"max-abs {np.abs(g['S'] - g32['S']).max():.2e}")
        assert max(errs) <= 1e-2
        assert rel_l2(g["S"], g32["S"]) <= 1e-2
        assert np.abs(g["S"] - g32["S"]).max() <= 2e-2
    # the FP32 form itself at the same voxels
    errs32 = [rel_l2(g32["E"][m][pts[:, 0], pts[:, 1], pts[:, 2]], Ec[:, m]) for m in range(3)]
    assert max(errs32) <= 1e-5, errs32


# ---- backward on the tensor cores ------------------------------------------------------------------

def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,shape,boundary,slabs", [
    (8, (7, 21, 37), "symmetric", 1),
    (8, (9, 16, 20), "zero", 3),
    (16, (6, 11, 35), "symmetric", 1),
    (16, (5, 9, 18), "periodic", 2),
])
def test_tensor_core_spectral_adjoint_matches_oracle(sal, prec, n, shape, boundary, slabs):
    V, _ = synth.volume(synth.small_spec(shape, seed=n + 3, faults=1))
    gE = synth.random_volume((3,) + shape, seed=n + 9)
    budget = 0
    if slabs > 1:
        # the backward's scratch: gE (3 planes), the reduction partials, and per t-plane of a slab the brick
        # blocks (n slices per brick, each XH x YH floats padded to a multiple of 4) plus one overlap-add plane
        # of brick slices; n - 1 more such planes are fixed.  The budget holds T // slabs planes of a slab.
        P = 128 // n
        nxs, nys = -(-shape[1] // P), -(-shape[2] // 16)
        slice_f = -(-(P + n - 1) * (16 + n - 1) // 4) * 4
        per_ext = nxs * nys * slice_f * 4
        per_t = n * per_ext
        base = sal.Saliency(shape, sal.Params(n=n, boundary=boundary, prec=prec))
        created = sal.sal_workspace_size(base.h)
        base.close()
        N = int(np.prod(shape))
        budget = (created + 3 * N * 4 + 1216 * 64 * 8 + (n - 1) * per_ext
                  + (per_t + per_ext) * max(1, shape[0] // slabs))
    eng = sal.Saliency(shape, sal.Params(n=n, boundary=boundary, prec=prec, hbm_budget_bytes=budget))
    try:
        gV = torch.empty(shape, dtype=torch.float32, device="cuda")
        sal.sal_local_spectra_project_backward(eng.h, _cuda(V), _cuda(gE), gV)
        torch.cuda.synchronize()
        got = gV.cpu().numpy()
    finally:
        eng.close()
    ref = oracle.features_adjoint(V, gE, n, boundary=boundary)
    err = rel_l2(got, ref)
    print(prec, n, shape, boundary, "gV rel-L2", f"{err:.2e}")
    assert err <= 1e-2


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,shape", [(8, (10, 18, 33)), (16, (6, 10, 20))])
def test_tensor_core_fused_backward(sal, prec, n, shape):
    V, D = synth.volume(synth.small_spec(shape, seed=n, faults=2))
    W = np.array([0.45, 0.35, 0.2])
    alpha = [1.0, 0.8, 1.2]
    params = sal.Params(n=n, alpha=alpha, prec=prec)
    st = oracle.dcs_stencil(params.directions, params.R, params.sigma, alpha)
    fwd = oracle.saliency(V, n, stencil=st, weights=W)
    gS = (fwd["S"] - D).astype(np.float32)
    ref = oracle.saliency_backward(V, n, W, gS, stencil=st, fwd=fwd)
    eng = sal.Saliency(shape, params)
    try:
        gV, gW, ga = eng.backward(_cuda(V), _cuda(W), _cuda(gS))
        torch.cuda.synchronize()
    finally:
        eng.close()
    errs = (rel_l2(gV.cpu().numpy(), ref["gV"]), rel_l2(gW.cpu().numpy(), ref["gW"]),
            rel_l2(ga.cpu().numpy(), ref["galpha"]))
    print(prec, n, shape, "gV gW galpha rel-L2", [f"{e:.2e}" for e in errs])
    assert max(errs) <= 1e-2


# ---- the 32^3 window -----------------------------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 1e-2), ("fp16", 1e-2)])
def test_window32_forward_matches_oracle(sal, prec, tol):
    shape = (5, 9, 21)
    V, _ = synth.volume(synth.small_spec(shape, seed=32, faults=2))
    p = sal.Params(n=32, prec=prec)
    g = _run(sal, V, p)
    ref = oracle.saliency(V, 32, stencil=oracle.dcs_stencil(p.directions, p.R, p.sigma))
    errs = {f"E{m}": rel_l2(g["E"][m], ref["E"][m]) for m in range(3)}
    errs.update({f"S{m}": rel_l2(g["S3"][m], ref["S3"][m]) for m in range(3)})
    errs["S"] = rel_l2(g["S"], ref["S"])
    print(prec, 32, shape, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= tol, (k, v)
    if prec != "fp32":
        assert np.abs(g["S"] - ref["S"]).max() <= 2e-2


@pytest.mark.parametrize("shape,taper", [((3, 4, 40), "rect"), ((3, 5, 19), "hann")])
def test_window32_fp32_sliding_and_taper(sal, shape, taper):
    """FP32, 32^3 window: rows of several y bricks (ragged last one) through the sliding form, and the Hann
    taper through the direct stage-3 sum."""
    V, _ = synth.volume(synth.small_spec(shape, seed=33, faults=2))
    g = _run(sal, V, sal.Params(n=32, taper=taper))
    E = oracle.features(V, 32, taper=taper)
    for m in range(3):
        assert rel_l2(g["E"][m], E[m]) <= 1e-5, (m, rel_l2(g["E"][m], E[m]))


def test_window32_constant_volume_gives_zero(sal):
    V = np.full((4, 5, 20), 1.75, np.float32)
    g = _run(sal, V, sal.Params(n=32))
    assert np.max(np.abs(g["E"])) <= 1e-5 * 1.75
    assert np.all(g["S"] == 0.0)


def test_window32_backward_is_not_built(sal):
    eng = sal.Saliency((4, 4, 8), sal.Params(n=32))
    try:
        with pytest.raises(sal.SalError) as ei:
            eng.backward(torch.zeros((4, 4, 8), device="cuda"), torch.ones(3, device="cuda") / 3,
                         torch.zeros((4, 4, 8), device="cuda"))
        assert ei.value.status == 2  # SAL_ERR_UNSUPPORTED
    finally:
        eng.close()
