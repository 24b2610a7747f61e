"""Parity at the largest workload: the 462 x 951 x 651 synthetic seismic volume (286 M voxels; 20 faults,
3 salt bodies, 4 channels), window 16, in the launch configuration the benchmark times.

E and the raw S_m come back from the device only at 44 seeded voxels and the 4 extreme corners, where the
FP64 oracle computes them one voxel at a time; the normalised map S is checked on the device by its
defining properties (min 0, max 1, and the min-max of the equal-weight sum of the min-max maps).
Tolerances as everywhere: FP32 relative L2 <= 1e-5 per map, the 16-bit tensor-core forms <= 1e-2.
The volume is generated once for all tests, its X slabs in parallel processes.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
SHAPE = (462, 951, 651)


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


@pytest.fixture(scope="module")
def volume():
    V, _ = synth.volume("full462x951x651", with_mask=False, workers=min(16, os.cpu_count() or 1))
    assert V.shape == SHAPE
    pts = np.concatenate([synth.sample_points(SHAPE, 44, seed=462),
                          [[0, 0, 0], [461, 950, 650], [0, 950, 325], [461, 0, 1]]])
    return V, pts


@pytest.mark.parametrize("prec,tol", [("bf16", 1e-2), ("fp32", 1e-5)])
def test_full_volume_forward_sampled(sal, volume, prec, tol):
    V, pts = volume
    p = sal.Params(n=16, prec=prec)
    eng = sal.Saliency(SHAPE, p)
    try:
        out = eng.saliency(torch.from_numpy(V).cuda(), None, intermediates=True)
        torch.cuda.synchronize()
        idx = torch.from_numpy(pts).cuda()
        Eg = out["E"][:, idx[:, 0], idx[:, 1], idx[:, 2]].T.cpu().numpy()
        Sg = out["S3"][:, idx[:, 0], idx[:, 1], idx[:, 2]].T.cpu().numpy()
        S, S3 = out["S"], out["S3"].double()
        lo = S3.amin(dim=(1, 2, 3)).view(3, 1, 1, 1)
        hi = S3.amax(dim=(1, 2, 3)).view(3, 1, 1, 1)
        C = ((S3 - lo) / (hi - lo)).mean(dim=0)
        Cn = (C - C.min()) / (C.max() - C.min())
        s_min, s_max = float(S.min()), float(S.max())
        s_err = float((S.double() - Cn).abs().max())
        del out, S, S3, C, Cn
    finally:
        eng.close()
    st = oracle.dcs_stencil(p.directions, p.R, p.sigma)
    Ec, Sc = oracle.center_surround_at(V, pts, 16, st[0], st[3])
    errs = [rel_l2(Eg[:, m], Ec[:, m]) for m in range(3)] + [rel_l2(Sg[:, m], Sc[:, m]) for m in range(3)]
    print(prec, "E, S_m sampled rel-L2", [f"{e:.2e}" for e in errs], "S property max-abs", f"{s_err:.1e}")
    assert max(errs) <= tol, errs
    assert s_min == 0.0 and abs(s_max - 1.0) <= 1e-6
    assert s_err <= 1e-5


def _adjoint_at(V, gEq, q):
    """The oracle's spectral adjoint gV[q] at interior voxels q, exactly: the windows that contain q are
    those centred at q - 7 .. q + 8 on each axis, all inside the 31^3 sub-volume around q, so the adjoint
    of that sub-volume with gE kept on those windows (zero elsewhere) gives gV[q]."""
    ref = []
    for (a, b, c), g in zip(q, gEq):
        gsub = np.zeros((3, 31, 31, 31))
        gsub[:, 8:24, 8:24, 8:24] = g
        ref.append(oracle.features_adjoint(V[a - 15:a + 16, b - 15:b + 16, c - 15:c + 16], gsub, 16)[15, 15, 15])
    return np.array(ref)


def sampled_spectral_adjoint(sal, V, prec, q, seed, with_ref=True):
    """gV of a seeded random gE from the library at voxels q, with the oracle's values there."""
    shape = V.shape
    gen = torch.Generator(device="cuda").manual_seed(seed)
    Vd = torch.from_numpy(V).cuda()
    gE = torch.randn((3,) + shape, device="cuda", generator=gen)
    eng = sal.Saliency(shape, sal.Params(n=16, prec=prec))
    try:
        gV = torch.empty(shape, device="cuda")
        sal.sal_local_spectra_project_backward(eng.h, Vd, gE, gV)
        qd = torch.from_numpy(q).cuda()
        got = gV[qd[:, 0], qd[:, 1], qd[:, 2]].cpu().numpy()
        gEq = [gE[:, a - 7:a + 9, b - 7:b + 9, c - 7:c + 9].cpu().numpy() for a, b, c in q]
    finally:
        eng.close()
    return got, (_adjoint_at(V, gEq, q) if with_ref else None)


def test_full_volume_spectral_adjoint(sal, volume):
    """The backward at full size, both forms against the oracle at 12 interior voxels (exact there, see
    _adjoint_at): FP32 at 1e-5, BF16 (the form the benchmark times; its adjoint's tensor-core operands
    are FP16) at 1e-2; and the whole BF16 gV against the FP32 one for the structured gradient gE = E."""
    V, _ = volume
    T, X, Y = SHAPE
    q = 15 + synth.sample_points((T - 31, X - 31, Y - 31), 12, seed=951)
    got32, ref = sampled_spectral_adjoint(sal, V, "fp32", q, 651)
    got16, _ = sampled_spectral_adjoint(sal, V, "bf16", q, 651, with_ref=False)
    err32, err16s = rel_l2(got32, ref), rel_l2(got16, ref)
    Vd = torch.from_numpy(V).cuda()
    eng = sal.Saliency(SHAPE, sal.Params(n=16, prec="fp32"))
    try:
        E = torch.empty((3,) + SHAPE, device="cuda")
        sal.sal_local_spectra_project(eng.h, Vd, E)
        gV32 = torch.empty(SHAPE, device="cuda")
        sal.sal_local_spectra_project_backward(eng.h, Vd, E, gV32)
        torch.cuda.synchronize()
    finally:
        eng.close()
    eng = sal.Saliency(SHAPE, sal.Params(n=16, prec="bf16"))
    try:
        gV16 = torch.empty(SHAPE, device="cuda")
        sal.sal_local_spectra_project_backward(eng.h, Vd, E, gV16)
        torch.cuda.synchronize()
        err16 = float((gV16.double() - gV32.double()).norm() / gV32.double().norm())
    finally:
        eng.close()
    print("spectral adjoint at 12 voxels vs oracle: FP32", f"{err32:.2e}", "BF16", f"{err16s:.2e}",
          "; BF16 vs FP32 whole volume", f"{err16:.2e}")
    assert err32 <= 1e-5 and err16s <= 1e-2 and err16 <= 1e-2


def test_salt128_spectral_adjoint_sampled(sal):
    """The 128^3 salt workload (window 16): both forms' spectral adjoint against the oracle at 12 interior
    voxels (exact there): FP32 at 1e-5, BF16 at 1e-2."""
    V, _ = synth.volume("salt128", with_mask=False)
    q = 15 + synth.sample_points((128 - 31,) * 3, 12, seed=128)
    got32, ref = sampled_spectral_adjoint(sal, V, "fp32", q, 128)
    got16, _ = sampled_spectral_adjoint(sal, V, "bf16", q, 128, with_ref=False)
    err32, err16 = rel_l2(got32, ref), rel_l2(got16, ref)
    print("salt128 spectral adjoint at 12 voxels vs oracle: FP32", f"{err32:.2e}", "BF16", f"{err16:.2e}")
    assert err32 <= 1e-5 and err16 <= 1e-2
