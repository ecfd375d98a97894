"""Many independent inversion problems at once: block products of uneven operators as
one CUDA graph or as one persistent kernel, and measured choices of engine, chunk, radix
order and tiles.

Each problem keeps its own operator (grid, kernel, spectra).  ``ProblemBatch.capture``
records every problem's G X and G^T Y into one CUDA graph, spreading the problems over
a few streams that fork from and join the capturing stream, so that problems too small
to fill the GPU run side by side and the whole batch costs one graph launch.
``NativeBatch`` binds the library's batch: ``products`` (forked streams, optionally one
recorded graph) and ``persistent`` (every problem's stages in one kernel launch over a
device-side work list, with bounded device waits).  ``tune`` picks engine, chunk and the
generic plans' radix orders per operator; ``tune_batch`` the persistent kernel's tiles.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional, Sequence, Tuple

import torch

__all__ = ["ProblemBatch", "NativeBatch", "tune", "tune_batch", "radix_orders", "TUNE_CACHE",
           "BATCH_TUNE_CACHE"]


class ProblemBatch:
    """Block products G_i X_i and G_i^T Y_i for operators ops[i], `columns` columns each."""

    def __init__(self, ops: Sequence, columns: int, streams: int = 8, seed: int = 0):
        self.ops = list(ops)
        self.columns = columns
        dev = self.ops[0].device
        gen = torch.Generator(device=dev).manual_seed(seed)
        self.X = [torch.randn(columns, op.n, generator=gen, device=dev, dtype=op.dtype)
                  for op in self.ops]
        self.Y = [torch.randn(columns, op.m, generator=gen, device=dev, dtype=op.dtype)
                  for op in self.ops]
        self.D = [torch.empty(columns, op.m, device=dev, dtype=op.dtype) for op in self.ops]
        self.XT = [torch.empty(columns, op.n, device=dev, dtype=op.dtype) for op in self.ops]
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(max(1, streams))]
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    @property
    def products(self) -> int:
        """Column products (G and G^T columns) per run of the batch."""
        return 2 * self.columns * len(self.ops)

    def _issue(self, forked: bool) -> None:
        main = torch.cuda.current_stream()
        if not forked:
            for i, op in enumerate(self.ops):
                op.matmat(self.X[i], out=self.D[i])
                op.rmatmat(self.Y[i], out=self.XT[i])
            return
        for s in self.streams:
            s.wait_stream(main)
        for i, op in enumerate(self.ops):
            with torch.cuda.stream(self.streams[i % len(self.streams)]):
                op.matmat(self.X[i], out=self.D[i])
                op.rmatmat(self.Y[i], out=self.XT[i])
        for s in self.streams:
            main.wait_stream(s)

    def run_eager(self, forked: bool = False) -> None:
        """One pass of all products launched directly (on one stream, or forked)."""
        self._issue(forked)

    def capture(self) -> None:
        """Record the forked batch into a CUDA graph (after an eager pass that sizes every
        operator's workspace, since no allocation may happen under capture)."""
        self._issue(True)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._issue(True)
        self.graph = g

    def replay(self) -> None:
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()


class NativeBatch:
    """The same batch through the C ABI (tf_batch_create / tf_batch_products): the library
    forks the operators' products over its own streams and, with use_graph, records them
    once as a CUDA graph and replays it while pointers and operator set-ups are unchanged."""

    def __init__(self, ops: Sequence, streams: int = 8):
        import ctypes
        from . import _lib
        self.ops = list(ops)
        self._ctypes, self._libm = ctypes, _lib
        arr = (ctypes.c_void_p * len(self.ops))(*[op._h for op in self.ops])
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().tf_batch_create(arr, len(self.ops), streams, ctypes.byref(h)))
        self._h = h

    def products(self, columns: int, X=None, D=None, Y=None, XT=None, use_graph: bool = True):
        """D[i] = G_i X[i] and XT[i] = G_i^T Y[i] (blocks of `columns` rows, row-major like
        Operator.matmat); None skips a direction."""
        ct = self._ctypes
        n = len(self.ops)

        def ptrs(ts):
            if ts is None:
                return None
            return (ct.c_void_p * n)(*[t.data_ptr() for t in ts])
        stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
        self._libm.check(self._libm.lib().tf_batch_products(
            self._h, columns, ptrs(X), ptrs(D), ptrs(Y), ptrs(XT), 1 if use_graph else 0, stream))

    def persistent(self, columns: int, X=None, D=None, Y=None, XT=None, rows_tile: int = 0,
                   cols_tile: int = 0, claim: int = 0, wait_ms: float = 0.0, gate=None,
                   use_graph: bool = False):
        """The same products as one persistent kernel launch (tf_batch_persistent); raises
        TFError with status TF_ETIMEOUT if a device-side wait ran out.  gate: an int32
        CUDA tensor that must become nonzero before the kernel starts work."""
        ct = self._ctypes
        n = len(self.ops)

        def ptrs(ts):
            if ts is None:
                return None
            return (ct.c_void_p * n)(*[t.data_ptr() for t in ts])
        opts = self._libm.tf_batch_opts(rows_tile, cols_tile, claim, float(wait_ms),
                                        gate.data_ptr() if gate is not None else None,
                                        1 if use_graph else 0)
        stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
        self._libm.check(self._libm.lib().tf_batch_persistent(
            self._h, columns, ptrs(X), ptrs(D), ptrs(Y), ptrs(XT), ct.byref(opts), stream))

    def close(self):
        if getattr(self, "_h", None):
            self._libm.lib().tf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# (n1, n2, nz, dtype, columns) -> (engine, chunk, x radices, y radices)
TUNE_CACHE: Dict[Tuple, Tuple] = {}
# (dtype, columns, problem shapes) -> (rows_tile, cols_tile) of the persistent batch kernel
BATCH_TUNE_CACHE: Dict[Tuple, Tuple[int, int]] = {}


def _time(fn, reps: int = 3) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def radix_orders(radices: Sequence[int], limit: int = 4) -> List[Tuple[int, ...]]:
    """Distinct orders of a radix multiset to try: the planner's own order, its reverse,
    the odd radices first, and a rotation (at most `limit`)."""
    base = tuple(radices)
    cands = [base, tuple(reversed(base)),
             tuple(sorted(base, key=lambda r: (r % 2 == 0, r))),
             base[1:] + base[:1]]
    out: List[Tuple[int, ...]] = []
    for c in cands:
        if c not in out:
            out.append(c)
    return out[:limit]


def tune(op, columns: int, chunks: Optional[List[int]] = None):
    """Measure G X + G^T Y on `columns` random columns and apply the fastest choice of
    engine (compile-time plans / generic), workspace chunk, and, for the generic engine,
    the radix order of each axis's plan; cached per (n1, n2, nz, dtype, columns).
    Returns (engine, chunk, x radices, y radices)."""
    key = (op.n1, op.n2, op.nz, str(op.dtype), columns)
    if key in TUNE_CACHE:
        engine, chunk, rx, ry = TUNE_CACHE[key]
        op.set_radices(0, rx)
        op.set_radices(1, ry)
        op.set_engine(engine)
        op.set_tuning(0, 0, chunk)
        return TUNE_CACHE[key]
    X = torch.randn(columns, op.n, device=op.device, dtype=op.dtype)
    Y = torch.randn(columns, op.m, device=op.device, dtype=op.dtype)
    chunks = chunks or sorted({max(1, columns // 4), max(1, columns // 2), columns})
    run = lambda: (op.matmat(X), op.rmatmat(Y))
    # radix orders of the generic engine, one axis at a time, at the largest chunk
    op.set_engine(1)
    op.set_tuning(0, 0, chunks[-1])
    best_r = []
    for axis in (0, 1):
        timed = []
        for order in radix_orders(op.radices(axis)):
            op.set_radices(axis, order)
            timed.append((_time(run), order))
        best_r.append(min(timed)[1])
        op.set_radices(axis, best_r[-1])
    best = None
    for engine in (0, 1):
        op.set_engine(engine)
        for chunk in chunks:
            op.set_tuning(0, 0, chunk)
            ms = _time(run)
            if best is None or ms < best[0]:
                best = (ms, engine, chunk)
    _, engine, chunk = best
    op.set_engine(engine)
    op.set_tuning(0, 0, chunk)
    TUNE_CACHE[key] = (engine, chunk, best_r[0], best_r[1])
    return TUNE_CACHE[key]


TILE_PAIRS = {torch.float32: [(8, 8), (16, 8), (8, 4), (4, 8)], torch.float64: [(4, 4), (8, 8)]}


def tune_batch(batch: "NativeBatch", columns: int, X, D, Y, XT, reps: int = 3):
    """Tile pair of the persistent batch kernel (sequence pairs per rows tile, k1 columns
    per column tile) measured on the batch's own products; applied through the returned
    (rows_tile, cols_tile) and cached per (dtype, columns, problem shapes)."""
    ops = batch.ops
    key = (str(ops[0].dtype), columns, tuple((op.n1, op.n2, op.nz) for op in ops))
    if key in BATCH_TUNE_CACHE:
        return BATCH_TUNE_CACHE[key]
    timed = []
    for tb, tk in TILE_PAIRS[ops[0].dtype]:
        ms = _time(lambda: batch.persistent(columns, X, D, Y, XT, rows_tile=tb, cols_tile=tk),
                   reps)
        timed.append((ms, (tb, tk)))
    BATCH_TUNE_CACHE[key] = min(timed)[1]
    return BATCH_TUNE_CACHE[key]
