"""Failure detection on the GPU, without a fault: a bounded device wait is made to give up.

The tensor-core kernels bound every mbarrier wait; a wait that gives up sets the handle's mapped error
word and its CTA leaves.  sal_check_bounded_wait runs that path on purpose (one CTA, an mbarrier that
no arrival completes, 1,000 tries).  The next call must return SAL_ERR_TIMEOUT, and the handle and the
CUDA context must then run a normal forward whose result matches the one before and the oracle."""
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


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_bounded_wait_gives_up_and_the_handle_recovers(sal, prec):
    shape = (12, 10, 37)
    V, _ = synth.volume(synth.small_spec(shape, seed=5, faults=1))
    Vt = torch.from_numpy(V).cuda()
    eng = sal.Saliency(shape, sal.Params(n=8, prec=prec))
    try:
        before = eng.local_spectra_project(Vt).cpu().numpy()
        sal.sal_check_bounded_wait(eng.h, 1000)
        torch.cuda.synchronize()
        with pytest.raises(sal.SalError) as ei:
            eng.local_spectra_project(Vt)
        assert ei.value.status == sal.SAL_ERR_TIMEOUT
        # the error word was cleared by the call that reported it: the next calls run normally
        after = eng.local_spectra_project(Vt).cpu().numpy()
        torch.cuda.synchronize()
        again = eng.saliency(Vt)["S"]
        torch.cuda.synchronize()
    finally:
        eng.close()
    assert np.array_equal(before, after)
    ref = oracle.features(V, 8)
    tol = 1e-5 if prec == "fp32" else 1e-2
    for m in range(3):
        assert np.linalg.norm(after[m] - ref[m]) <= tol * np.linalg.norm(ref[m])
    assert torch.isfinite(again).all()


def test_bounded_wait_argument_check(sal):
    eng = sal.Saliency((8, 8, 8), sal.Params(n=8))
    try:
        with pytest.raises(sal.SalError) as ei:
            sal.sal_check_bounded_wait(eng.h, 0)
        assert ei.value.status == sal.SAL_ERR_INVALID_ARG
    finally:
        eng.close()
