"""GPU parity of the 2-D section mode against the oracle's 2-D definition.  A section is passed as a
volume one sample thick with symmetric or periodic extension (every cube is then constant across the
section, so only the in-plane DFT remains):

  * a vertical section [T][X] (time x crossline) as [T][X][1], the default t, x, t-x window, weights
    (1/2, 1/2, 0): the library's E_t, E_x are the section's two projected features and E_y its
    unprojected mean abs(F_2D);
  * a time slice [X][Y] as [1][X][Y], an in-plane x, y, x-y window, weights (0, 1/2, 1/2).

Tolerances as for volumes: FP32 relative L2 <= 1e-5; BF16 / FP16 relative L2 <= 1e-2 per map and
max-abs <= 2e-2 on S.
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


def _reference(A, n, boundary, vertical, directions, W):
    """The 2-D method on section A from the oracle's 2-D definition, in the library's map order."""
    Es = oracle.section_features(A, n, boundary)            # [E_0 (unprojected), E_a, E_b]
    E = np.stack([Es[1], Es[2], Es[0]])[..., None] if vertical else Es[:, None]
    offs, g, did, w = oracle.dcs_stencil(directions, 3, 1.5)
    S3 = oracle.center_surround(E, offs, w, boundary)
    out = oracle.combine(S3, np.asarray(W, float))
    out.update({"E": E, "S3": S3})
    return out


@pytest.mark.parametrize("vertical", [True, False])
@pytest.mark.parametrize("n,shape,boundary,prec,tol", [
    (8, (40, 37), "symmetric", "fp32", 1e-5),
    (16, (33, 50), "periodic", "fp32", 1e-5),
    (8, (40, 37), "symmetric", "bf16", 1e-2),
    (16, (33, 50), "symmetric", "fp16", 1e-2),
])
def test_section_matches_2d_definition(sal, vertical, n, shape, boundary, prec, tol):
    V, _ = synth.volume(synth.small_spec(shape + (6,) if vertical else (6,) + shape, seed=n + shape[0], faults=2))
    A = np.ascontiguousarray(V[:, :, 3] if vertical else V[3])
    vol = A[:, :, None] if vertical else A[None]
    directions = ((1, 0, 0), (0, 1, 0), (1, 1, 0)) if vertical else ((0, 1, 0), (0, 0, 1), (0, 1, 1))
    W = (0.5, 0.5, 0.0) if vertical else (0.0, 0.5, 0.5)
    ref = _reference(A, n, boundary, vertical, directions, W)
    p = sal.Params(n=n, boundary=boundary, prec=prec, directions=directions, R=3)
    eng = sal.Saliency(vol.shape, p)
    try:
        out = eng.saliency(torch.from_numpy(np.ascontiguousarray(vol)).cuda(), None,
                           torch.tensor(W, dtype=torch.float32, device="cuda"), intermediates=True)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        eng.close()
    errs = {f"E{m}": rel_l2(g["E"][m], ref["E"][m]) for m in range(3)}
    errs.update({f"S{m}": rel_l2(g["S3"][m], ref["S3"][m]) for m in range(3)})
    errs["S"] = rel_l2(g["S"], ref["S"])
    print(prec, n, shape, boundary, "vertical" if vertical else "slice", {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= tol, (k, v)
    if prec != "fp32":
        assert np.abs(g["S"] - ref["S"]).max() <= 2e-2
