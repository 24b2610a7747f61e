"""Pins of the oracle's stride-s windows (cubes only at voxels whose indices are multiples of s, the
features interpolated in between) against facts fixed by the definition:

  * on the lattice the stride-s features are the stride-1 features of the same voxels, exactly;
  * the interpolation reproduces an affine field exactly up to the last lattice point of each axis
    and holds that point's value beyond it;
  * one unit lattice value spreads as the separable tent (1 - |d_t|/s)(1 - |d_x|/s)(1 - |d_y|/s);
  * stride 1 is the per-voxel definition itself.
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
