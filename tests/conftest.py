import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(autouse=True)
def _bounds_record(request):
    """With TF_LIB_VARIANT=checked (bounds-checked library), fail any GPU test whose
    kernels recorded an out-of-bounds access."""
    yield
    import os
    if os.environ.get("TF_LIB_VARIANT") != "checked" or "gpu" not in request.keywords:
        return
    import ctypes
    import torch
    from paper_2004_13904_gb300 import _lib
    torch.cuda.synchronize()
    c, s, o, e = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    _lib.lib().tf_debug_oob(ctypes.byref(c), ctypes.byref(s), ctypes.byref(o), ctypes.byref(e))
    assert c.value == 1, "TF_LIB_VARIANT=checked but the library is not a checked build"
    assert s.value == 0, f"out-of-bounds access: site {s.value}, offset {o.value}, extent {e.value}"
