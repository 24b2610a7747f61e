"""GPU parity of the center-surround step (Eq. 3) and its adjoint with a richer directional template
than the default three lines of Fig. 4: all 13 directions of the 3x3x3 neighbourhood (one per
antipodal pair), two steps each way (52 neighbours), per-direction weights alpha_d.

Tolerance (FP32 path): relative L2 <= 1e-5.  Both sides take the same FP32 features and the
kernel's FP32 weights w_o = alpha_d g_o, so every sign of a difference is decided on identical
numbers.  The volumes are wider than 128 along y, so the row loops run more than one chunk, and
thin enough along t and x that border and interior voxels both occur.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RTOL = 1e-5

DIRS13 = tuple(d for d in itertools.product((-1, 0, 1), repeat=3)
               if d != (0, 0, 0) and next(c for c in d if c != 0) > 0)


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


@pytest.mark.parametrize("shape,boundary", [((10, 9, 140), "symmetric"), ((8, 7, 133), "periodic"),
                                            ((7, 10, 150), "zero"), ((12, 26, 140), "symmetric")])
def test_13_direction_template_forward_and_adjoint(sal, shape, boundary):
    V, _ = synth.volume(synth.small_spec(shape, seed=sum(shape), faults=1))
    E32 = oracle.features(V, 4, boundary=boundary).astype(np.float32)
    gS3 = synth.random_volume((3,) + shape, seed=17)
    alpha = np.linspace(0.6, 1.4, len(DIRS13))
    params = sal.Params(n=4, boundary=boundary, directions=DIRS13, R=2, alpha=alpha)
    offs, g, did, _ = oracle.dcs_stencil(DIRS13, 2, 1.5, alpha)
    assert len(DIRS13) == 13 and not {tuple(-c for c in d) for d in DIRS13} & set(DIRS13)
    assert len(offs) == 52
    w32 = (alpha.astype(np.float32)[did] * g.astype(np.float32)).astype(np.float64)   # the kernel's weights
    eng = sal.Saliency(shape, params)
    try:
        S3 = torch.empty((3,) + shape, dtype=torch.float32, device="cuda")
        sal.sal_center_surround(eng.h, _cuda(E32), S3)
        gE = torch.empty((3,) + shape, dtype=torch.float32, device="cuda")
        ga = torch.empty(len(DIRS13), dtype=torch.float32, device="cuda")
        sal.sal_center_surround_backward(eng.h, _cuda(E32), _cuda(gS3), gE, ga)
        torch.cuda.synchronize()
    finally:
        eng.close()
    ref3 = oracle.center_surround(E32, offs, w32, boundary=boundary)
    for m in range(3):
        assert rel_l2(S3[m].cpu().numpy(), ref3[m]) <= RTOL, (m, rel_l2(S3[m].cpu().numpy(), ref3[m]))
    refE, gw = oracle.center_surround_adjoint(E32, gS3, offs, w32, boundary)
    ref_ga = oracle.direction_gradient(gw, g.astype(np.float32), did)
    assert rel_l2(gE.cpu().numpy(), refE) <= RTOL, rel_l2(gE.cpu().numpy(), refE)
    assert rel_l2(ga.cpu().numpy(), ref_ga) <= RTOL, rel_l2(ga.cpu().numpy(), ref_ga)
