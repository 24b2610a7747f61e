"""Pins of the oracle's stride-s windows (cubes only at voxels whose indices are multiples of s, the
features interpolated in between) against facts fixed by the definition:

  * on the lattice the stride-s features are the stride-1 features of the same voxels, exactly;
  * the interpolation reproduces an affine field exactly up to the last lattice point of each axis
    and holds that point's value beyond it;
  * one unit lattice value spreads as the separable tent (1 - |d_t|/s)(1 - |d_x|/s)(1 - |d_y|/s);
  * stride 1 is the per-voxel definition itself;
  * the interpolation's adjoint satisfies <upsample(a), b> = <a, upsample_adjoint(b)>, and the
    stride-s feature adjoint matches central differences of the stride-s features (the energy
    feature: a quadratic form, so the differences are exact up to rounding).
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n,s,boundary,feature", [(4, 1, "symmetric", "abs"), (8, 2, "symmetric", "abs"),
                                                  (8, 3, "periodic", "energy"), (16, 4, "zero", "abs")])
def test_lattice_values_are_the_per_voxel_features(n, s, boundary, feature):
    V = synth.random_volume((11, 9, 14), seed=n + s)
    Es = oracle.features(V, n, boundary=boundary, feature=feature, stride=s)
    E1 = oracle.features(V, n, boundary=boundary, feature=feature)
    assert Es.shape == E1.shape
    lat = np.ix_(range(3), range(0, 11, s), range(0, 9, s), range(0, 14, s))
    assert np.array_equal(Es[lat], E1[lat])
    if s == 1:
        assert np.array_equal(Es, E1)


@pytest.mark.parametrize("s,shape", [(2, (9, 7, 10)), (3, (10, 8, 13)), (4, (5, 9, 12))])
def test_upsample_reproduces_affine_fields(s, shape):
    Tc, Xc, Yc = (-(-d // s) for d in shape)
    tc, xc, yc = np.meshgrid(np.arange(Tc) * s, np.arange(Xc) * s, np.arange(Yc) * s, indexing="ij")
    coef = np.array([[0.5, -1.25, 2.0, 0.75], [3.0, 0.1, -0.2, 0.3], [-1.0, 0.0, 0.0, 1.0]])
    Ec = np.stack([c[0] + c[1] * tc + c[2] * xc + c[3] * yc for c in coef])
    E = oracle.upsample(Ec, s, shape)
    t, x, y = np.meshgrid(*(np.minimum(np.arange(d), s * (-(-d // s) - 1)) for d in shape), indexing="ij")
    ref = np.stack([c[0] + c[1] * t + c[2] * x + c[3] * y for c in coef])
    assert np.allclose(E, ref, rtol=0, atol=1e-12)


def test_upsample_of_one_lattice_value_is_the_tent():
    s, shape = 3, (13, 10, 11)
    Tc, Xc, Yc = (-(-d // s) for d in shape)
    Ec = np.zeros((3, Tc, Xc, Yc))
    a = (2, 1, 2)                                  # lattice point (6, 3, 6), away from the last ones
    Ec[1][a] = 1.0
    E = oracle.upsample(Ec, s, shape)
    hat = [np.maximum(0.0, 1.0 - np.abs(np.arange(d) - s * c) / s) for d, c in zip(shape, a)]
    ref = hat[0][:, None, None] * hat[1][None, :, None] * hat[2][None, None, :]
    assert np.allclose(E[1], ref, atol=1e-15) and not E[0].any() and not E[2].any()


@pytest.mark.parametrize("s,shape", [(2, (9, 7, 10)), (3, (10, 8, 13))])
def test_upsample_adjoint_dot_product(s, shape):
    rng = np.random.default_rng(s)
    Tc, Xc, Yc = (-(-d // s) for d in shape)
    a = rng.standard_normal((3, Tc, Xc, Yc))
    b = rng.standard_normal((3,) + shape)
    lhs = np.sum(oracle.upsample(a, s, shape) * b)
    rhs = np.sum(a * oracle.upsample_adjoint(b, s))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("boundary", ["symmetric", "periodic"])
def test_stride_feature_adjoint_matches_exact_differences(boundary):
    n, s = 8, 3
    V = synth.random_volume((8, 7, 10), seed=31).astype(np.float64)
    gE = synth.random_volume((3,) + V.shape, seed=32).astype(np.float64)
    gV = oracle.features_adjoint(V, gE, n, boundary=boundary, feature="energy", stride=s)
    eps = 1e-3
    for p in synth.sample_points(V.shape, 10, seed=4).tolist() + [[0, 0, 0], [7, 6, 9]]:
        Vp = V.copy(); Vp[tuple(p)] += eps
        Vm = V.copy(); Vm[tuple(p)] -= eps
        fd = (np.sum(gE * oracle.features(Vp, n, boundary=boundary, feature="energy", stride=s))
              - np.sum(gE * oracle.features(Vm, n, boundary=boundary, feature="energy", stride=s))) / (2 * eps)
        # exact for a quadratic form; the bound is the rounding of the two O(1e3) sums differenced
        assert abs(fd - gV[tuple(p)]) <= 1e-7 * max(1.0, abs(fd)), (p, fd, gV[tuple(p)])
