"""GPU parity of the forward path (FP32 form) against the FP64 oracle, through the C ABI.

Tolerance (FP32 path): relative L2 error <= 1e-5 per map (E_t, E_x, E_y, S_t, S_x, S_y, S).
Inputs are the seeded synthetic volumes shared with the oracle; sizes span several CTA
bricks with ragged tails in y, and the small worked examples of the oracle pins.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_F32 = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


@pytest.fixture(scope="module")
def sal():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_06174_gb300 as s
    s.load()
    return s


def _window(params):
    """The oracle's own window for the same directions, R, sigma and alpha."""
    if params.offsets is None:
        return oracle.dcs_stencil(params.directions, params.R, params.sigma, params.alpha)
    offs = np.asarray(params.offsets, np.int32).reshape(-1, 3)
    g = np.asarray(params.gauss_w, np.float64)
    did = np.asarray(params.dir_id, np.int32)
    alpha = np.ones(did.max() + 1) if params.alpha is None else np.asarray(params.alpha, float)
    return offs, g, did, alpha[did] * g


def _run(sal, V, params, D=None, W=None):
    eng = sal.Saliency(V.shape, params)
    try:
        out = eng.saliency(torch.from_numpy(V).cuda(), None if D is None else torch.from_numpy(D).cuda(),
                           None if W is None else torch.tensor(W, dtype=torch.float32).cuda(), intermediates=True)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        eng.close()


@pytest.mark.parametrize("n,shape,boundary", [
    (2, (5, 7, 40), "symmetric"),
    (4, (9, 6, 45), "periodic"),
    (4, (7, 8, 33), "zero"),
    (8, (12, 10, 70), "symmetric"),
    (8, (6, 11, 37), "zero"),
    (16, (8, 7, 37), "symmetric"),
    (16, (5, 6, 20), "periodic"),
])
def test_features_match_oracle(sal, n, shape, boundary):
    V, _ = synth.volume(synth.small_spec(shape, seed=n + shape[2], faults=1))
    p = sal.Params(n=n, boundary=boundary)
    g = _run(sal, V, p)
    E = oracle.features(V, n, boundary=boundary)
    for m in range(3):
        assert rel_l2(g["E"][m], E[m]) <= RTOL_F32, (m, rel_l2(g["E"][m], E[m]))
    st = _window(p)
    S3 = oracle.center_surround(E, st[0], st[3], boundary=boundary)
    for m in range(3):
        assert rel_l2(g["S3"][m], S3[m]) <= RTOL_F32, (m, rel_l2(g["S3"][m], S3[m]))
    ref = oracle.combine(S3, "equal")
    assert rel_l2(g["S"], ref["S"]) <= RTOL_F32


@pytest.mark.parametrize("n,prec,tol", [(8, "fp32", RTOL_F32), (16, "fp32", RTOL_F32), (8, "bf16", 1e-2),
                                         (16, "fp16", 1e-2)])
def test_hann_taper_features_match_oracle(sal, n, prec, tol):
    """The periodic Hann taper on every axis of the cube.  In the FP32 form it keeps the direct stage-3
    sum (the sliding recursion along y holds for the rect cube only), so both forms are covered."""
    shape = (7, 9, 37)
    V, _ = synth.volume(synth.small_spec(shape, seed=n + 7, faults=1))
    g = _run(sal, V, sal.Params(n=n, taper="hann", prec=prec))
    E = oracle.features(V, n, taper="hann")
    for m in range(3):
        assert rel_l2(g["E"][m], E[m]) <= tol, (m, rel_l2(g["E"][m], E[m]))


@pytest.mark.parametrize("n,shape", [(8, (4, 5, 200)), (16, (3, 4, 150))])
def test_sliding_form_long_rows(sal, n, shape):
    """Rows long enough for many y bricks (ragged last brick): every chunk of the sliding recursion
    restarts from a direct sum, so the error stays at the level of the direct form."""
    V, _ = synth.volume(synth.small_spec(shape, seed=n + 11, faults=2))
    g = _run(sal, V, sal.Params(n=n))
    E = oracle.features(V, n)
    for m in range(3):
        assert rel_l2(g["E"][m], E[m]) <= RTOL_F32, (m, rel_l2(g["E"][m], E[m]))


def test_fault48_n8_whole_volume(sal):
    """The 48^3 fault volume, window 8, every map element by element."""
    V, D = synth.volume("fault48")
    p = sal.Params(n=8)
    st = _window(p)
    ref = oracle.saliency(V, 8, stencil=st)
    g = _run(sal, V, p)
    for m in range(3):
        assert rel_l2(g["E"][m], ref["E"][m]) <= RTOL_F32
        assert rel_l2(g["S3"][m], ref["S3"][m]) <= RTOL_F32
    assert rel_l2(g["S"], ref["S"]) <= RTOL_F32
    # template-fitted weights (LS, FP64 sums on the device)
    refD = oracle.combine(ref["S3"], "ls", D)
    gD = _run(sal, V, p, D=D)
    assert np.allclose(gD["W"], refD["W"], rtol=1e-4, atol=1e-5)
    assert rel_l2(gD["S"], refD["S"]) <= RTOL_F32
    # given weights
    W = [0.2, 0.5, 0.3]
    gW = _run(sal, V, p, W=W)
    refW = oracle.combine(ref["S3"], np.array(W))
    assert rel_l2(gW["S"], refW["S"]) <= RTOL_F32
    assert np.allclose(gW["W"], W)


def test_salt128_n16_sampled(sal):
    """128^3 salt/fold/fault volume, window 16: raw E and S_m at 48 seeded voxels computed one
    by one by the oracle; the normalised map checked by its defining properties."""
    V, _ = synth.volume("salt128")
    p = sal.Params(n=16)
    g = _run(sal, V, p)
    st = _window(p)
    pts = np.concatenate([synth.sample_points(V.shape, 44, seed=77), [[0, 0, 0], [127, 127, 127], [0, 127, 64],
                                                                     [127, 0, 3]]])
    Ec, Sc = oracle.center_surround_at(V, pts, 16, st[0], st[3])
    Eg = g["E"][:, pts[:, 0], pts[:, 1], pts[:, 2]].T
    Sg = g["S3"][:, pts[:, 0], pts[:, 1], pts[:, 2]].T
    for m in range(3):
        assert rel_l2(Eg[:, m], Ec[:, m]) <= RTOL_F32
        assert rel_l2(Sg[:, m], Sc[:, m]) <= RTOL_F32
    S = g["S"]
    assert S.min() == 0.0 and abs(S.max() - 1.0) <= 1e-6
    # S is the min-max of the equal-weight sum of the min-max maps of S3 (property at any size)
    S3 = g["S3"].astype(np.float64)
    Shat = np.stack([(S3[m] - S3[m].min()) / (S3[m].max() - S3[m].min()) for m in range(3)])
    C = Shat.mean(axis=0)
    assert np.max(np.abs(S - (C - C.min()) / (C.max() - C.min()))) <= 1e-5


def test_worked_example_on_gpu(sal):
    from conftest import load_golden
    gold = load_golden("impulse_4x4x4_n2.txt")
    V = np.zeros((4, 4, 4), np.float32)
    V[1, 1, 1] = 1.0
    offs = np.array([[-1, 0, 0], [1, 0, 0]])
    p = sal.Params(n=2, boundary="periodic", offsets=offs, gauss_w=np.full(2, np.exp(-0.5)), dir_id=[0, 0])
    g = _run(sal, V, p)
    inner = np.zeros((4, 4, 4), bool)
    inner[1:3, 1:3, 1:3] = True
    cap = np.zeros((4, 4, 4), bool)
    cap[[0, 3], 1:3, 1:3] = True
    for m in range(3):
        assert np.allclose(g["E"][m][inner], gold["c2"], atol=2e-7)
        assert np.all(np.abs(g["E"][m][~inner]) <= 1e-7)
        assert np.allclose(g["S3"][m][inner], gold["S_inner"], atol=2e-7)
        assert np.allclose(g["S3"][m][cap], gold["S_cap"], atol=2e-7)
    assert np.allclose(g["S"][cap], gold["S_norm_cap"], atol=1e-6)
    assert np.allclose(g["S"][inner], 1.0, atol=1e-6)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_constant_volume_gives_zero(sal, n):
    V = np.full((9, 10, 19), -2.5, np.float32)
    g = _run(sal, V, sal.Params(n=n))
    assert np.max(np.abs(g["E"])) <= 1e-5 * 2.5
    assert np.all(g["S"] == 0.0)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 2), (2, 1, 17), (3, 2, 1)])
def test_degenerate_tiny_volumes(sal, shape):
    """Windows much larger than the volume: the symmetric extension repeats the volume."""
    V = synth.random_volume(shape, seed=sum(shape))
    for n in (4, 8):
        g = _run(sal, V, sal.Params(n=n, R=1))
        E = oracle.features(V, n)
        # a 1x1x1 volume extends to a constant: E is 0 up to rounding on both sides, so the
        # relative error is replaced by an absolute floor of FP32 rounding of |V|
        floor = 1e-6 * np.abs(V).max() * np.sqrt(V.size)
        for m in range(3):
            err = np.linalg.norm(g["E"][m].astype(np.float64) - E[m])
            assert err <= RTOL_F32 * np.linalg.norm(E[m]) + floor


def test_deterministic(sal):
    V, D = synth.volume(synth.small_spec((16, 12, 50), seed=3, faults=2))
    a = _run(sal, V, sal.Params(n=8), D=D)
    b = _run(sal, V, sal.Params(n=8), D=D)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_stepwise_calls_match_fused(sal):
    V, D = synth.volume(synth.small_spec((10, 9, 35), seed=4, faults=1))
    p = sal.Params(n=8)
    eng = sal.Saliency(V.shape, p)
    try:
        Vt = torch.from_numpy(V).cuda()
        E = eng.local_spectra_project(Vt)
        S3 = eng.center_surround(E)
        S, W = eng.combine(S3, D=torch.from_numpy(D).cuda())
        fused = eng.saliency(Vt, D=torch.from_numpy(D).cuda(), intermediates=True)
        torch.cuda.synchronize()
        assert torch.equal(E, fused["E"]) and torch.equal(S3, fused["S3"])
        assert torch.equal(S, fused["S"]) and torch.equal(W, fused["W"])
    finally:
        eng.close()


def test_error_paths(sal):
    p = sal.Params(n=8, hbm_budget_bytes=1024)
    with pytest.raises(sal.SalError) as ei:
        sal.Saliency((16, 16, 16), p)
    assert ei.value.status == 3  # SAL_ERR_OOM
    eng = sal.Saliency((8, 8, 8), sal.Params(n=8))
    try:
        with pytest.raises(sal.SalError) as ei:
            sal.sal_local_spectra_project(eng.h, None, None)
        assert ei.value.status == 1
    finally:
        eng.close()
