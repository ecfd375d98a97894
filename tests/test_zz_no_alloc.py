"""tf_matvec_noalloc: the forward product for callers that cannot allocate device memory
when they run it (it uses the library's fixed scratch buffer instead of the operator's
workspace).  Checked against tf_matvec on two calls in a row, through the C ABI.

This file is collected last on purpose: it runs after every other test when the whole
suite runs, and it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-5, "f64": 1e-12}


def _call(L, op, x, d, cs=None, rs=None):
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.tf_matvec_noalloc(op._h, ptr(x), ptr(d), ptr(cs), ptr(rs), stream)


@pytest.mark.parametrize("dtn", ["f32", "f64"])
def test_noalloc_matches_matvec_twice(dtn):
    import torch
    from paper_2004_13904_gb300 import Operator, _lib
    dt = torch.float32 if dtn == "f32" else torch.float64
    L = _lib.lib()
    g = synth.config_grid("c2")
    op = Operator(g, "gravity", dtype=dt)
    rng = np.random.default_rng(42)
    for call in range(2):                   # the second call reuses the shared scratch
        x = torch.tensor(rng.standard_normal(g.n), dtype=dt, device="cuda")
        cs = torch.tensor(rng.uniform(0.5, 2.0, g.n), dtype=dt, device="cuda")
        rs = torch.tensor(rng.uniform(0.5, 2.0, g.m), dtype=dt, device="cuda")
        ref = op.matvec(x, colscale=cs, rowscale=rs)
        d = torch.full((g.m,), float("nan"), dtype=dt, device="cuda")
        assert _call(L, op, x, d, cs, rs) == _lib.TF_OK, L.tf_last_error()
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(d - ref) / torch.linalg.norm(ref))
        assert err <= TOL[dtn], (call, err)
    op.close()


def test_noalloc_rejects_oversize_problem():
    import torch
    from paper_2004_13904_gb300 import Operator, _lib
    L = _lib.lib()
    g = synth.config_grid("c4")              # 9.1 MB of FP32 scratch per column > 8 MiB
    op = Operator(g, "gravity", dtype=torch.float32)
    x = torch.zeros(g.n, device="cuda")
    d = torch.zeros(g.m, device="cuda")
    assert _call(L, op, x, d) == _lib.TF_EINVAL
    assert "scratch" in L.tf_last_error().decode()
    op.close()
