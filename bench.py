"""Benchmark of the BTTB/BCCB block products on GB300.

Workload (one "step"): the c2 gravity problem -- 100 x 100 stations over a
110 x 110 x 10 volume of 50 m cubes (5 % padding per side; m = 10000, n = 121000) --
with one block product G X and one transpose block product G^T Y on 1260 FP32 columns
each (the RSVD block size k+p = 1250+10).  Metric: column products per second
(G and G^T columns), whole job.  Inputs (610 MB + 50 MB) exceed the 126 MB L2, so
no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f32|f64] [--impl reference]

Under torchrun each rank runs its own 1260-column block (weak scaling, no collective on
the data path); the timed region is bracketed by a barrier and synchronisation and the
maximum over ranks is reported.  --impl reference times the FP64 CPU oracle (numpy FFT
route) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

CONFIG = "c2"
BLOCK = 1260
WORKLOAD = ("c2 gravity: 100x100 stations, 110x110x10 cells of 50 m (5% padding), "
            "m=10000, n=121000; G X and G^T Y on 1260 columns per step")

# DRAM traffic per launch of the dominant kernel from an ncu capture, keyed by the
# hash of the kernel sources at capture time (null once the kernels change).
# cols_fwd, c2, FP32: 313.2 MB (DRAM read 292.7 + write 20.5) for one 256-column launch,
# scaled to the benchmark's 1260-column launch by columns (traffic grows in proportion).
NCU_TRAFFIC = {
    ("cols_fwd", "c2", "f32"): {"hash": "9a66cb5ead2e3134", "bytes_per_launch": 313.2e6 * 1260 / 256},
}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("tf_ct_kernels.cuh", "tf_fft_ct.cuh", "tf_fft.cuh", "tf_check.cuh"):
        with open(os.path.join(ROOT, "paper_2004_13904_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def fp32_peak_tflops(sm_mhz: float) -> float:
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def fft_flops(n: int) -> float:
    return 5.0 * n * math.log2(n) if n > 1 else 0.0


def stage_model(g):
    """Algorithmic flops and bytes per column of each stage, at the minimum embedding
    (sx+nx-1) x (sy+ny-1) of App. A (a larger FFT size chosen by the library is a cost,
    not extra credit).  FFT flops: 5 N log2 N per complex transform of length N; two real
    rows share one complex transform."""
    n1, n2 = g.n1min, g.n2min
    nh = n1 // 2 + 1
    rows_m = g.nz * g.ny
    cols = {
        "rows_r2c_model": (rows_m / 2 * fft_flops(n1), 4 * g.n + 8 * rows_m * nh),
        "cols_fwd": ((g.nz + 1) * nh * fft_flops(n2) + 8 * g.nz * nh * n2,
                     8 * rows_m * nh + 8 * g.sy * nh),
        "rows_c2r_data": (g.sy / 2 * fft_flops(n1), 8 * g.sy * nh + 4 * g.m),
        "rows_r2c_data": (g.sy / 2 * fft_flops(n1), 4 * g.m + 8 * g.sy * nh),
        "cols_adj": ((g.nz + 1) * nh * fft_flops(n2) + 6 * g.nz * nh * n2,
                     8 * g.sy * nh + 8 * rows_m * nh),
        "rows_c2r_model": (rows_m / 2 * fft_flops(n1), 8 * rows_m * nh + 4 * g.n),
    }
    return cols


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(g, seconds: float = 12.0):
    """FP64 numpy oracle (FFT route, as it stands) on columns of the same workload."""
    from oracle import operator as oop
    T = oop.layer_tables(g, "gravity")
    X = synth.gaussian_columns(g.n, 2, seed=123)
    Y = synth.gaussian_columns(g.m, 2, seed=321)
    t0 = time.perf_counter()
    done = 0
    while True:
        oop.fft_matvec(g, T, X[done % 2])
        oop.fft_rmatvec(g, T, Y[done % 2])
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return 2 * done / dt, 2 * done, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g = synth.config_grid(CONFIG)
    from oracle import operator as oop
    T = oop.layer_tables(g, "gravity")
    X = synth.gaussian_columns(g.n, 4, seed=123)
    Y = synth.gaussian_columns(g.m, 4, seed=321)
    per_step = 4

    def step():
        for b in range(per_step):
            oop.fft_matvec(g, T, X[b])
            oop.fft_rmatvec(g, T, Y[b])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = 2 * per_step * args.steps / dt
    sample = f"{per_step} G and {per_step} G^T columns per step (of {BLOCK})"
    print(json.dumps({
        "impl": "reference", "metric": "G/G^T column products per second", "value": value,
        "unit": "products/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "block_columns": per_step, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "products/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="column chunks of the host-buffer pipeline (Operator.products_host)")
    ap.add_argument("--columns", type=int, default=BLOCK,
                    help="columns per block (default: the 1260-column RSVD block); smaller "
                         "blocks serve profiling captures")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2004_13904_gb300 import Operator, STAGES, peak_tflops
    from paper_2004_13904_gb300.parallel import max_over_ranks

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    dt = torch.float32 if args.dtype == "f32" else torch.float64
    g = synth.config_grid(CONFIG)
    op = Operator(g, "gravity", dtype=dt)
    dev = torch.device("cuda", local)
    cols_per_rank = args.columns
    X = torch.tensor(synth.gaussian_columns(g.n, cols_per_rank, seed=123 + rank), dtype=dt, device=dev)
    Y = torch.tensor(synth.gaussian_columns(g.m, cols_per_rank, seed=321 + rank), dtype=dt, device=dev)
    D = torch.empty((cols_per_rank, g.m), dtype=dt, device=dev)
    XT = torch.empty((cols_per_rank, g.n), dtype=dt, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        op.matmat(X, out=D)
        op.rmatmat(Y, out=XT)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    op.profile(True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = op.profile_read()
    op.profile(False)
    ms = max_over_ranks(ms, dev)
    products = 2 * cols_per_rank * args.steps * world
    value = products / (ms / 1e3)

    # end to end through the public API with pinned host buffers
    esz = 4 if dt == torch.float32 else 8
    e2e = None
    if args.e2e_steps > 0:
        Xh = X.cpu().pin_memory()
        Yh = Y.cpu().pin_memory()
        Dh = torch.empty((cols_per_rank, g.m), dtype=dt, pin_memory=True)
        XTh = torch.empty((cols_per_rank, g.n), dtype=dt, pin_memory=True)
        op.products_host(Xh, Yh, Dh, XTh, chunks=args.e2e_chunks)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            op.products_host(Xh, Yh, Dh, XTh, chunks=args.e2e_chunks)
            torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        barrier()
        e2e_s = max_over_ranks(e2e_s, dev)
        e2e = {"value": 2 * cols_per_rank * args.e2e_steps * world / e2e_s, "unit": "products/s",
               "h2d_bytes_per_step": (g.n + g.m) * cols_per_rank * esz,
               "d2h_bytes_per_step": (g.m + g.n) * cols_per_rank * esz}

    # roofline of the dominant kernel, timed live with events on the launching stream
    model = stage_model(g)
    top = max(STAGES, key=lambda s: prof[s][0])
    tms, launches, cols = prof[top]
    flops, bytes_ = model[top]
    per_launch_cols = cols / max(launches, 1)
    avg_s = tms / 1e3 / max(launches, 1)
    pk, pk_kind = peaks()
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    measured = peak_tflops(dt)
    achieved = flops * per_launch_cols / avg_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": measured, "unit": "TFLOP/s",
            "frac": achieved / measured,
            "peak_source": f"measured: FMA-chain probe in {args.dtype} on this GPU"
                           + (f"; derived FP32 peak 152 SMs x 128 lanes x 2 x {sm_max:.0f} MHz "
                              f"= {fp32_peak_tflops(sm_max):.1f}" if dt == torch.float32 else ""),
            "hbm": {"achieved_gbs": bytes_ * per_launch_cols / avg_s / 1e9,
                    "peak_gbs": pk["hbm_gbs"], "peak_source": f"hbm_gbs ({pk_kind})"}}
    tr = NCU_TRAFFIC.get((top, CONFIG, args.dtype))
    ok = tr and tr["hash"] == kernel_hash() and cols_per_rank == BLOCK
    roof["traffic"] = tr["bytes_per_launch"] if ok else None
    roof["kernel"] = top
    roof["launch_ms"] = avg_s * 1e3
    roof["columns_per_launch"] = per_launch_cols
    stage_share = {s: prof[s][0] / max(sum(v[0] for v in prof.values()), 1e-30) for s in STAGES}
    hbm_alg = (esz * g.n + esz * g.m) * 2 * cols_per_rank * args.steps / (ms / 1e3) / 1e9
    gpu_launches = int(sum(v[1] for v in prof.values()))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": "G/G^T column products per second", "value": value, "unit": "products/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "block_columns": cols_per_rank, "fft": [op.n1, op.n2],
                   "tuning": list(op.tuning()),
                   "l2": (f"inputs (X {g.n * cols_per_rank * esz / 1e6:.0f} MB, "
                          f"Y {g.m * cols_per_rank * esz / 1e6:.0f} MB) "
                          + ("exceed L2; no flush" if g.n * cols_per_rank * esz > 129e6 else
                             "fit in L2"))},
        "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roof,
        "hbm_algorithmic_gbs": hbm_alg, "stage_share": stage_share, "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        rate, ncols, secs = cpu_oracle_rate(g)
        line["cpu_baseline"] = {"value": rate, "unit": "products/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"{ncols} FP64 column products (numpy FFT route) in "
                                          f"{secs:.1f} s; host has {os.cpu_count()} cores"}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
