"""sal_combine_noalloc: the combination step for callers that cannot allocate device memory
(a caller-owned pool or arena, a region that forbids allocation).  Its scratch is a static
device array shared by all calls.  This file sorts last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_noalloc_combine_matches_handle_combine_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_06174_gb300 as sal
    cases = [((20, 18, 41), True, None), ((11, 9, 50), False, [0.2, 0.5, 0.3])]
    for k, (shape, with_D, W) in enumerate(cases):
        V, D = synth.volume(synth.small_spec(shape, seed=30 + k, faults=2))
        eng = sal.Saliency(shape, sal.Params(n=8))
        try:
            E = eng.local_spectra_project(torch.from_numpy(V).cuda())
            S3 = eng.center_surround(E)
            Dt = torch.from_numpy(D).cuda() if with_D else None
            Wt = torch.tensor(W, dtype=torch.float32).cuda() if W is not None else None
            S_ref, W_ref = eng.combine(S3, D=Dt, W=Wt)
            S_na = torch.full_like(S_ref, float("nan"))
            W_na = torch.full((3,), float("nan"), device=S_ref.device)
            sal.sal_combine_noalloc(S3, Dt, Wt, W_na, S_na)
            torch.cuda.synchronize()
            assert rel_l2(S_na, S_ref) <= 1e-5
            assert torch.allclose(W_na, W_ref, rtol=1e-5, atol=1e-6)
        finally:
            eng.close()


def test_noalloc_equal_weights_and_large_volume_twice():
    """Equal weights (D and W_in both NULL), and a volume of about 4.2 M voxels, where the noalloc grid
    (one partial slot per 4,096 voxels) differs most from sal_combine's; two calls in a row each."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_06174_gb300 as sal
    g = torch.Generator(device="cuda").manual_seed(7)
    for shape, with_D in [((13, 10, 47), False), ((96, 211, 207), False), ((96, 211, 207), True)]:
        S3 = torch.rand((3,) + shape, device="cuda", generator=g)
        Dt = (torch.rand(shape, device="cuda", generator=g) > 0.8).float() if with_D else None
        eng = sal.Saliency(shape, sal.Params(n=8))
        try:
            S_ref, W_ref = eng.combine(S3, D=Dt)
            for _ in range(2):
                S_na = torch.full_like(S_ref, float("nan"))
                W_na = torch.full((3,), float("nan"), device=S_ref.device)
                sal.sal_combine_noalloc(S3, Dt, None, W_na, S_na)
                torch.cuda.synchronize()
                assert rel_l2(S_na, S_ref) <= 1e-5
                assert torch.allclose(W_na, W_ref, rtol=1e-5, atol=1e-6)
        finally:
            eng.close()


def test_noalloc_rejects_buffers_off_the_current_device():
    """A host buffer where device memory is expected is refused before any work."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    import paper_2201_06174_gb300 as sal
    L = sal.load()
    host = (ctypes.c_float * (3 * 8))()
    S = torch.empty((2, 2, 2), device="cuda")
    st = L.sal_combine_noalloc(2, 2, 2, ctypes.cast(host, ctypes.c_void_p), None, None, 1e-6, None,
                               ctypes.c_void_p(S.data_ptr()), None)
    assert st == 1  # SAL_ERR_INVALID_ARG
    assert "S3" in sal.sal_last_error_text(None)


def test_noalloc_rejects_volumes_beyond_the_static_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_06174_gb300 as sal
    L = sal.load()
    st = L.sal_combine_noalloc(257, 256, 256, None, None, None, 1e-6, None, None, None)
    assert st == 2  # SAL_ERR_UNSUPPORTED, before any device work
    assert "16777216" in sal.sal_last_error_text(None)
