"""The persistent batch kernel (tf_batch_persistent) on the fifth configuration's uneven
problems at their real sizes (32-128 stations per side, 8-16 layers, 0-10 % padding, half
magnetic): bitwise equal to each operator's own generic-engine products (same stage code,
same tiles and plans), per-problem parity with the FP64 oracle, graph replay, a device-side
wait that runs out (a start gate nothing opens) reported as TF_ETIMEOUT with the context
still usable, and the tuners."""
import numpy as np
import pytest

import synth
from oracle import operator as oop

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-5, "f64": 1e-12}


def _dt(dtn):
    import torch
    return torch.float32 if dtn == "f32" else torch.float64


def _ops(dtn, idx):
    from paper_2004_13904_gb300 import Operator
    probs = synth.batch_problems(64, seed=5)
    return [Operator(probs[i].grid, probs[i].kind, probs[i].inc, probs[i].dec, dtype=_dt(dtn))
            for i in idx], [probs[i] for i in idx]


def _blocks(ops, cols, seed, dtn):
    import torch
    gen = torch.Generator(device="cuda").manual_seed(seed)
    X = [torch.randn(cols, op.n, generator=gen, device="cuda", dtype=_dt(dtn)) for op in ops]
    Y = [torch.randn(cols, op.m, generator=gen, device="cuda", dtype=_dt(dtn)) for op in ops]
    D = [torch.full((cols, op.m), float("nan"), device="cuda", dtype=_dt(dtn)) for op in ops]
    XT = [torch.full((cols, op.n), float("nan"), device="cuda", dtype=_dt(dtn)) for op in ops]
    return X, Y, D, XT


@pytest.mark.parametrize("dtn,tiles", [("f32", (8, 8)), ("f32", (16, 8)), ("f64", (4, 4))])
def test_persistent_bitwise_equals_single_generic_products(dtn, tiles):
    import torch
    from paper_2004_13904_gb300.batch import NativeBatch
    ops, _ = _ops(dtn, range(0, 64, 4))           # 16 of the 64 problems, every size class
    for op in ops:
        op.set_engine(1)                             # the generic engine, as the kernel runs
        op.set_tuning(tiles[0], tiles[1], 0)
    cols = 3
    X, Y, D, XT = _blocks(ops, cols, 1, dtn)
    ref_D = [op.matmat(x) for op, x in zip(ops, X)]
    ref_XT = [op.rmatmat(y) for op, y in zip(ops, Y)]
    b = NativeBatch(ops)
    b.persistent(cols, X, D, Y, XT, rows_tile=tiles[0], cols_tile=tiles[1])
    torch.cuda.synchronize()
    for a, r in zip(D + XT, ref_D + ref_XT):
        assert torch.equal(a, r)
    b.close()


def test_persistent_matches_oracle_per_problem():
    """A third of the 64 problems, FP32, both directions, every column against the
    oracle's FFT route; plus one direction only (G^T Y) for the same batch."""
    import torch
    from paper_2004_13904_gb300.batch import NativeBatch
    idx = list(range(0, 64, 3))
    ops, probs = _ops("f32", idx)
    cols = 2
    X, Y, D, XT = _blocks(ops, cols, 2, "f32")
    b = NativeBatch(ops)
    b.persistent(cols, X, D, Y, XT)
    torch.cuda.synchronize()
    worst = 0.0
    for i, (op, p) in enumerate(zip(ops, probs)):
        T = oop.layer_tables(p.grid, p.kind, p.inc, p.dec)
        for c in range(cols):
            x = X[i][c].double().cpu().numpy()
            y = Y[i][c].double().cpu().numpy()
            rd = oop.fft_matvec(p.grid, T, x)
            rx = oop.fft_rmatvec(p.grid, T, y)
            e1 = np.linalg.norm(D[i][c].double().cpu().numpy() - rd) / np.linalg.norm(rd)
            e2 = np.linalg.norm(XT[i][c].double().cpu().numpy() - rx) / np.linalg.norm(rx)
            worst = max(worst, e1, e2)
    print(f"persistent batch, {len(ops)} problems: worst rel err {worst:.2e}")
    assert worst <= TOL["f32"]
    XT2 = [torch.full_like(t, float("nan")) for t in XT]
    b.persistent(cols, Y=Y, XT=XT2)
    torch.cuda.synchronize()
    assert all(torch.equal(a, r) for a, r in zip(XT2, XT))
    b.close()


def test_persistent_graph_replay():
    import torch
    from paper_2004_13904_gb300.batch import NativeBatch
    ops, _ = _ops("f32", range(1, 64, 8))
    cols = 4
    X, Y, D, XT = _blocks(ops, cols, 3, "f32")
    b = NativeBatch(ops)
    b.persistent(cols, X, D, Y, XT)
    torch.cuda.synchronize()
    ref = [t.clone() for t in D + XT]
    for _ in range(3):                      # eager with the graph's key, record + launch, replay
        for t in D + XT:
            t.fill_(float("nan"))
        b.persistent(cols, X, D, Y, XT, use_graph=True)
        torch.cuda.synchronize()
        assert all(torch.equal(a, r) for a, r in zip(D + XT, ref))
    b.close()


def test_persistent_wait_times_out_and_context_survives():
    """A start gate that nothing sets: every CTA's bounded wait runs out after about 20 ms,
    the kernel records TF_ETIMEOUT and returns; the same batch then runs normally."""
    import torch
    from paper_2004_13904_gb300 import _lib
    from paper_2004_13904_gb300.batch import NativeBatch
    ops, _ = _ops("f32", range(2, 64, 16))
    cols = 2
    X, Y, D, XT = _blocks(ops, cols, 4, "f32")
    ref_D = [op.matmat(x) for op, x in zip(ops, X)]
    b = NativeBatch(ops)
    gate = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(_lib.TFError) as e:
        b.persistent(cols, X, D, Y, XT, wait_ms=20.0, gate=gate)
    assert e.value.status == _lib.TF_ETIMEOUT
    gate.fill_(1)                            # an opened gate lets the same launch through
    b.persistent(cols, X, D, Y, XT, wait_ms=20.0, gate=gate)
    b.persistent(cols, X, D, Y, XT)
    torch.cuda.synchronize()
    for op, d, r in zip(ops, D, ref_D):
        assert float(torch.linalg.norm(d - r) / torch.linalg.norm(r)) <= TOL["f32"]
    b.close()


def test_tuners_keep_results():
    import torch
    from paper_2004_13904_gb300 import _lib
    from paper_2004_13904_gb300.batch import NativeBatch, TILE_PAIRS, radix_orders, tune_batch
    ops, _ = _ops("f32", range(5, 64, 12))
    cols = 2
    X, Y, D, XT = _blocks(ops, cols, 5, "f32")
    b = NativeBatch(ops)
    b.persistent(cols, X, D, Y, XT)
    torch.cuda.synchronize()
    ref = [t.clone() for t in D + XT]
    pair = tune_batch(b, cols, X, D, Y, XT)
    assert pair in TILE_PAIRS[torch.float32]
    op = ops[0]
    for axis in (0, 1):
        for order in radix_orders(op.radices(axis)):
            op.set_radices(axis, order)
            assert op.radices(axis) == tuple(order)
    b.persistent(cols, X, D, Y, XT, rows_tile=pair[0], cols_tile=pair[1])
    torch.cuda.synchronize()
    for a, r in zip(D + XT, ref):
        assert float(torch.linalg.norm(a - r) / torch.linalg.norm(r)) <= TOL["f32"]
    with pytest.raises(_lib.TFError):
        op.set_radices(0, (3, 3))            # product is not the length
    with pytest.raises(_lib.TFError):
        b.persistent(cols, X, D, Y, XT, rows_tile=16, cols_tile=16)   # pair not compiled
    b.close()
