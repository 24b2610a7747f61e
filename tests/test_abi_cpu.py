"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports every
entry point include/sal.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2201_06174_gb300 as sal
from paper_2201_06174_gb300 import sal as salmod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "sal.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:sal_status|const char\s*\*)\s*(sal_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_entry_points():
    assert _declared() == sorted(sal.ENTRY_POINTS)


def test_library_exports_every_declared_symbol():
    L = sal.load()
    for name in _declared():
        assert hasattr(L, name), name


def _create(**kw):
    p = sal.Params(**{k: v for k, v in kw.items() if k in sal.Params.__dataclass_fields__})
    shape = kw.get("shape", (8, 8, 8))
    return sal.sal_create(p, shape)


@pytest.mark.parametrize("kw,status", [
    (dict(n=3), salmod.SAL_ERR_INVALID_ARG),
    (dict(n=0), salmod.SAL_ERR_INVALID_ARG),
    (dict(n=34), salmod.SAL_ERR_INVALID_ARG),
    (dict(n=6), salmod.SAL_ERR_UNSUPPORTED),
    (dict(n=32, prec="bf16", shape=(70000, 4, 4)), salmod.SAL_ERR_UNSUPPORTED),
    (dict(shape=(0, 4, 4)), salmod.SAL_ERR_INVALID_ARG),
    (dict(shape=(70000, 4, 4)), salmod.SAL_ERR_UNSUPPORTED),
    (dict(offsets=np.array([[9, 0, 0]]), gauss_w=np.array([1.0]), dir_id=np.array([0])), salmod.SAL_ERR_INVALID_ARG),
    (dict(offsets=np.array([[1, 0, 0]]), gauss_w=np.array([np.nan]), dir_id=np.array([0])), salmod.SAL_ERR_INVALID_ARG),
    (dict(alpha=[np.inf, 1, 1]), salmod.SAL_ERR_INVALID_ARG),
    (dict(ls_delta=-1.0), salmod.SAL_ERR_INVALID_ARG),
    # the spatial-domain reading of the feature step: FP32, n in {2, 4, 8, 16}, stride 1
    (dict(n=8, feature="spatial", prec="bf16"), salmod.SAL_ERR_UNSUPPORTED),
    (dict(n=32, feature="spatial"), salmod.SAL_ERR_UNSUPPORTED),
    (dict(n=8, feature="spatial", stride=2), salmod.SAL_ERR_UNSUPPORTED),
])
def test_create_rejects_bad_arguments_before_device_work(kw, status):
    with pytest.raises(sal.SalError) as ei:
        _create(**kw)
    assert ei.value.status == status
    assert sal.sal_last_error_text(None) != ""


def test_null_params_and_out():
    L = sal.load()
    h = ctypes.c_void_p()
    assert L.sal_create(None, 4, 4, 4, ctypes.byref(h)) == salmod.SAL_ERR_INVALID_ARG
    p = salmod.sal_params()
    assert L.sal_create(ctypes.byref(p), 4, 4, 4, None) == salmod.SAL_ERR_INVALID_ARG


def test_null_handle_calls():
    L = sal.load()
    for name, nargs in [("sal_local_spectra_project", 4), ("sal_center_surround", 4), ("sal_combine", 7),
                        ("sal_saliency", 9), ("sal_saliency_backward", 8), ("sal_local_spectra_project_backward", 5),
                        ("sal_center_surround_backward", 6), ("sal_combine_backward", 7)]:
        assert getattr(L, name)(*([None] * nargs)) == salmod.SAL_ERR_INVALID_ARG
    assert L.sal_check_bounded_wait(None, 1, None) == salmod.SAL_ERR_INVALID_ARG
    assert L.sal_destroy(None) == salmod.SAL_OK
    assert L.sal_workspace_size(None, None) == salmod.SAL_ERR_INVALID_ARG


def test_product_window_matches_oracle_window():
    """The product and the oracle build the Fig. 4 window independently; they must agree."""
    import oracle
    offs, g, did = sal.directional_window()
    o2, g2, d2, w2 = oracle.dcs_stencil()
    assert np.array_equal(offs, o2) and np.array_equal(did, d2)
    assert np.allclose(g, g2, rtol=1e-7)


def test_library_window_argument_checks():
    """sal_directional_window (host only) rejects bad radii, sigmas, zero directions, neighbours beyond
    +-8 and windows larger than the capacity."""
    L = sal.load()
    ip = ctypes.POINTER(ctypes.c_int)
    offs = np.zeros((64, 3), np.int32)
    g = np.zeros(64, np.float32)
    did = np.zeros(64, np.int32)
    q = ctypes.c_int()

    def call(dirs, R, sigma, cap=64):
        d = np.ascontiguousarray(dirs, np.int32).reshape(-1, 3)
        return L.sal_directional_window(len(d), d.ctypes.data_as(ip), R, sigma, cap, ctypes.byref(q),
                                        offs.ctypes.data_as(ip), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        did.ctypes.data_as(ip))
    assert call([[1, 0, 0]], 3, 1.5) == salmod.SAL_OK and q.value == 6
    assert call([[1, 0, 0]], 0, 1.5) == salmod.SAL_ERR_INVALID_ARG
    assert call([[1, 0, 0]], 2, 0.0) == salmod.SAL_ERR_INVALID_ARG
    assert call([[1, 0, 0]], 2, float("nan")) == salmod.SAL_ERR_INVALID_ARG
    assert call([[0, 0, 0]], 2, 1.0) == salmod.SAL_ERR_INVALID_ARG
    assert call([[3, 0, 0]], 3, 1.0) == salmod.SAL_ERR_INVALID_ARG        # 9 > 8
    assert call([[1, 0, 0]] * 11, 3, 1.0) == salmod.SAL_ERR_INVALID_ARG   # 66 > 64
    assert call([[1, 0, 0]], 3, 1.5, cap=5) == salmod.SAL_ERR_INVALID_ARG
    # the default (NULL directions) is the three directions of Fig. 4
    assert L.sal_directional_window(0, None, 3, 1.5, 64, ctypes.byref(q), offs.ctypes.data_as(ip),
                                    g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), did.ctypes.data_as(ip)) == 0
    import oracle
    o2, g2, d2, _ = oracle.dcs_stencil()
    assert q.value == len(g2) and np.array_equal(offs[:q.value], o2) and np.array_equal(did[:q.value], d2)
    assert np.allclose(g[:q.value], g2, rtol=1e-7)


@pytest.mark.parametrize("dirs,R,sigma", [(((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)), 2, 0.8),
                                         (((0, 1, 0), (0, 0, 1), (0, 1, 1)), 3, 1.5),
                                         (((1, -1, 0), (2, 0, 1)), 4, 2.5)])
def test_library_window_matches_oracle_window_any_directions(dirs, R, sigma):
    import oracle
    offs, g, did = sal.directional_window(dirs, R, sigma)
    o2, g2, d2, _ = oracle.dcs_stencil(dirs, R, sigma)
    assert np.array_equal(offs, o2) and np.array_equal(did, d2)
    assert np.allclose(g, g2, rtol=1e-7)
