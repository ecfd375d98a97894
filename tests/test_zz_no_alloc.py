"""tf_matvec_noalloc: the forward product for callers that cannot allocate device memory
when they run it (it uses the library's fixed scratch buffer instead of the operator's
workspace).  Checked against tf_matvec on two calls in a row, against the FP64 oracle
after a larger operator has left its data in the shared scratch, and for the device's
free memory, which must not change across the calls -- the first call on a fresh
operator included.

This file is collected last on purpose: it runs after every other test when the whole
suite runs, and it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import operator as oop

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-5, "f64": 1e-12}


def _call(L, op, x, d, cs=None, rs=None):
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.tf_matvec_noalloc(op._h, ptr(x), ptr(d), ptr(cs), ptr(rs), stream)


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]          # cudaMemGetInfo: the device's free bytes


@pytest.mark.parametrize("dtn", ["f32", "f64"])
def test_noalloc_matches_matvec_twice(dtn):
    import torch
    from paper_2004_13904_gb300 import Operator, _lib
    dt = torch.float32 if dtn == "f32" else torch.float64
    L = _lib.lib()
    g = synth.config_grid("c2")
    op = Operator(g, "gravity", dtype=dt)
    assert op.engine() == (0, True, True)    # compiled plans for tf_matvec; the call runs generic
    rng = np.random.default_rng(42)
    xs = [torch.tensor(rng.standard_normal(g.n), dtype=dt, device="cuda") for _ in range(2)]
    css = [torch.tensor(rng.uniform(0.5, 2.0, g.n), dtype=dt, device="cuda") for _ in range(2)]
    rss = [torch.tensor(rng.uniform(0.5, 2.0, g.m), dtype=dt, device="cuda") for _ in range(2)]
    outs = [torch.full((g.m,), float("nan"), dtype=dt, device="cuda") for _ in range(2)]
    # the operator's very first product is the allocation-free one: nothing may allocate
    free0 = _free_bytes()
    for call in range(2):                   # the second call reuses the shared scratch
        assert _call(L, op, xs[call], outs[call], css[call], rss[call]) == _lib.TF_OK, L.tf_last_error()
        assert _free_bytes() == free0, call
    for call in range(2):
        ref = op.matvec(xs[call], colscale=css[call], rowscale=rss[call])
        err = float(torch.linalg.norm(outs[call] - ref) / torch.linalg.norm(ref))
        assert err <= TOL[dtn], (call, err)
    op.close()


@pytest.mark.parametrize("dtn", ["f32", "f64"])
def test_noalloc_after_larger_operator_matches_oracle(dtn):
    """A larger operator fills more of the shared scratch first; the smaller one's result
    must not depend on what is left there.  Both are checked against the FP64 oracle."""
    import torch
    from paper_2004_13904_gb300 import Operator, _lib
    dt = torch.float32 if dtn == "f32" else torch.float64
    L = _lib.lib()
    big = synth.config_grid("c2")
    small = synth.padded_grid(37, 23, 5, 0.08)
    rng = np.random.default_rng(7)
    cases = []
    for g, kind, inc, dec in ((big, "gravity", 90.0, 0.0), (small, "magnetic", 60.0, 15.0),
                              (big, "gravity", 90.0, 0.0)):
        op = Operator(g, kind, inc, dec, dtype=dt)
        x = rng.standard_normal(g.n)
        d = torch.full((g.m,), float("nan"), dtype=dt, device="cuda")
        cases.append((g, kind, inc, dec, op, x, torch.tensor(x, dtype=dt, device="cuda"), d))
    free0 = _free_bytes()
    for g, kind, inc, dec, op, x, xd, d in cases:
        assert _call(L, op, xd, d) == _lib.TF_OK, L.tf_last_error()
    assert _free_bytes() == free0
    for g, kind, inc, dec, op, x, xd, d in cases:
        ref = oop.fft_matvec(g, oop.layer_tables(g, kind, inc, dec), x)
        got = d.double().cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL[dtn], (g, err)
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
