"""The C ABI library builds, loads, exports every declared entry point, and rejects bad
arguments on the host (no GPU needed: every case fails before any CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2004_13904_gb300 import build, _lib
    build.build()
    return _lib.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:tf_status|const char\*)\s+(tf_\w+)\s*\(", text, re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_header():
    from paper_2004_13904_gb300 import _lib
    names = set(declared_symbols()) - {"tf_last_error"}
    assert names <= set(_lib.SIGNATURES), names - set(_lib.SIGNATURES)


def _grid(**kw):
    from paper_2004_13904_gb300 import _lib
    import synth
    g = synth.Grid(4, 3, 2)
    s, keep = _lib.make_grid(g)
    for k, v in kw.items():
        setattr(s, k, v)
    return s, keep


@pytest.mark.parametrize("field,value", [("sx", 0), ("nz", 0), ("pxl", -1), ("dx", 0.0),
                                         ("station_z", 10.0)])
def test_create_rejects_bad_geometry(L, field, value):
    from paper_2004_13904_gb300 import _lib
    g, keep = _grid(**{field: value})
    h = ctypes.c_void_p(123)
    st = L.tf_create_gravity(ctypes.byref(g), _lib.TF_F32, None, ctypes.byref(h))
    assert st == _lib.TF_EINVAL
    assert h.value is None
    assert L.tf_last_error().decode()


def test_create_rejects_nonincreasing_z(L):
    from paper_2004_13904_gb300 import _lib
    g, keep = _grid()
    keep[1] = keep[0]
    h = ctypes.c_void_p()
    assert L.tf_create_magnetic(ctypes.byref(g), 50.0, 10.0, 5e4, _lib.TF_F64, None,
                                ctypes.byref(h)) == _lib.TF_EINVAL
    assert "increasing" in L.tf_last_error().decode()


def test_create_rejects_bad_dtype_and_null(L):
    from paper_2004_13904_gb300 import _lib
    g, keep = _grid()
    h = ctypes.c_void_p()
    assert L.tf_create_gravity(ctypes.byref(g), 7, None, ctypes.byref(h)) == _lib.TF_EINVAL
    assert L.tf_create_gravity(None, _lib.TF_F32, None, ctypes.byref(h)) == _lib.TF_EINVAL
    assert L.tf_create_gravity(ctypes.byref(g), _lib.TF_F32, None, None) == _lib.TF_EINVAL


def test_null_operator_rejected(L):
    from paper_2004_13904_gb300 import _lib
    m = ctypes.c_int64()
    assert L.tf_dims(None, ctypes.byref(m), None) == _lib.TF_EINVAL
    assert L.tf_matvec(None, None, None, None, None, None) == _lib.TF_EINVAL
    assert L.tf_rmatmat(None, 1, None, 1, None, 1, None, None, None) == _lib.TF_EINVAL
    assert L.tf_destroy(None) == _lib.TF_OK
