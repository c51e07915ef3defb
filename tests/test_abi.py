"""C ABI checks that need no GPU: the library loads, exports every symbol include/pff.h declares,
and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1902_08112_gb300 import pff

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "pff.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pff_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pff.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return pff.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in pff.SIGNATURES, n


def test_default_params(lib):
    p = pff.default_params()
    assert (p.E, p.nu, p.Gc, p.kappa, p.c_as, p.tol_as) == (1.0, 0.2, 1.0, 1e-10, 100.0, 1e-10)
    assert (p.mg_precision, p.cheb_degree, p.cg_steps, p.coarse_maxit, p.seed) == (32, 4, 10, 200, 12345)
    assert (p.tie_scale, p.newton_rtol, p.coarse_phi_max, p.split, p.preconditioner) == (0, 1e-8, 0, 0, 0)


@pytest.mark.parametrize("field,value", [("dim", 4), ("degree", 3), ("n_levels", 0)])
def test_create_rejects_bad_mesh(lib, field, value):
    m = pff.make_mesh(3, 1, (8, 8, 8), 2, (-1,) * 3, (1,) * 3)
    setattr(m, field, value)
    h = ctypes.c_void_p()
    st = lib.pff_create_hierarchy(ctypes.byref(m), ctypes.byref(pff.default_params()), None, ctypes.byref(h))
    assert st == pff.EINVAL and not h.value


def test_create_rejects_indivisible_levels(lib):
    m = pff.make_mesh(2, 1, (12, 12), 4, (-1, -1), (1, 1))     # 12 not divisible by 8
    h = ctypes.c_void_p()
    st = lib.pff_create_hierarchy(ctypes.byref(m), ctypes.byref(pff.default_params()), None, ctypes.byref(h))
    assert st == pff.EINVAL


def test_create_rejects_bad_params(lib):
    m = pff.make_mesh(2, 1, (8, 8), 2, (-1, -1), (1, 1))
    h = ctypes.c_void_p()
    for kw in ({"mg_precision": 16}, {"eps": 0.0}, {"nu": 0.5}, {"cg_steps": 0}, {"tie_scale": 2},
               {"newton_rtol": 0.0}, {"coarse_phi_max": 2}):
        st = lib.pff_create_hierarchy(ctypes.byref(m), ctypes.byref(pff.default_params(**kw)), None,
                                      ctypes.byref(h))
        assert st == pff.EINVAL


def test_null_handle_calls(lib):
    assert lib.pff_destroy_hierarchy(None) == pff.OK
    assert lib.pff_apply_jacobian(None, 0, None, None) == pff.EINVAL
    assert lib.pff_last_error(None) == b"null hierarchy"
