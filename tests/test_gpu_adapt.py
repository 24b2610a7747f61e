"""The paper's adaptive weight update (LMS, NLMS, RLS) on the GPU against the FP64 oracle's
sequential filters, per block of inline sections, and RLS against the least-squares fit."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sal():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_06174_gb300 as s
    s.load()
    return s


@pytest.fixture(scope="module")
def maps(sal):
    V, D = synth.volume(synth.small_spec((12, 10, 16), seed=3, faults=1))
    eng = sal.Saliency(V.shape, sal.Params(n=8))
    try:
        out = eng.saliency(torch.from_numpy(V).cuda(), None, intermediates=True)
        torch.cuda.synchronize()
        S3 = out["S3"].cpu().numpy()
    finally:
        eng.close()
    return V.shape, S3, D.astype(np.float32)


def _oracle_blocks(S3, D, method, sections):
    S3d = S3.astype(np.float64)
    lo = S3d.reshape(3, -1).min(1)
    hi = S3d.reshape(3, -1).max(1)
    Shat = np.stack([oracle.minmax(S3d[m], lo[m], hi[m]) for m in range(3)])
    Y = S3.shape[3]
    sec = sections if sections > 0 else Y
    Ws, tr = [], []
    for y0 in range(0, Y, sec):
        W, e2 = oracle.adapt_weights(Shat[:, :, :, y0:y0 + sec], D[:, :, y0:y0 + sec], method=method, return_trace=True)
        Ws.append(W)
        tr.append(e2)
    return np.array(Ws), np.concatenate(tr)


@pytest.mark.parametrize("method", ["lms", "nlms", "rls"])
@pytest.mark.parametrize("sections", [0, 4])
def test_adaptive_weights_match_oracle(sal, maps, method, sections):
    shape, S3, D = maps
    eng = sal.Saliency(shape, sal.Params(n=8))
    try:
        nblk = 1 if sections == 0 else -(-shape[2] // sections)
        W = torch.empty((nblk, 3), dtype=torch.float32, device="cuda")
        err2 = torch.empty(int(np.prod(shape)), dtype=torch.float32, device="cuda")
        sal.sal_adapt_weights(eng.h, torch.from_numpy(S3).cuda(), torch.from_numpy(D).cuda(), W, method=method,
                              sections=sections, err2=err2)
        torch.cuda.synchronize()
        Wg, eg = W.cpu().numpy().astype(np.float64), err2.cpu().numpy().astype(np.float64)
    finally:
        eng.close()
    Wo, eo = _oracle_blocks(S3, D, method, sections)
    werr = np.abs(Wg - Wo).max() / max(np.abs(Wo).max(), 1e-30)
    terr = np.linalg.norm(eg - eo) / max(np.linalg.norm(eo), 1e-30)
    print(method, sections, "W rel", f"{werr:.2e}", "err^2 trace rel-L2", f"{terr:.2e}")
    # the GPU normalises the maps with an FP32 reciprocal of (max - min): ~1e-7 relative in x
    assert werr <= 1e-5, (Wg, Wo)
    assert terr <= 1e-4


def test_rls_reaches_the_least_squares_fit(sal, maps):
    """RLS with lambda = 1 and P0 = I/delta is the ridge least-squares solution (G + delta I)^-1 b that
    sal_combine fits from the same desired map."""
    shape, S3, D = maps
    eng = sal.Saliency(shape, sal.Params(n=8))
    try:
        S3d, Dd = torch.from_numpy(S3).cuda(), torch.from_numpy(D).cuda()
        W_rls = torch.empty((1, 3), dtype=torch.float32, device="cuda")
        sal.sal_adapt_weights(eng.h, S3d, Dd, W_rls, method="rls")
        W_ls = torch.empty(3, dtype=torch.float32, device="cuda")
        S = torch.empty(shape, dtype=torch.float32, device="cuda")
        sal.sal_combine(eng.h, S3d, Dd, None, W_ls, S)
        torch.cuda.synchronize()
    finally:
        eng.close()
    a, b = W_rls.cpu().numpy()[0], W_ls.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-4 * max(1.0, np.abs(b).max()), (a, b)
