"""Benchmark of the BTTB/BCCB block products on GB300.

Workload (one "step", default): the c4 gravity problem at paper scale -- 250 x 200 stations
over a 250 x 200 x 20 volume of 50 m cubes (m = 50 000, n = 1 000 000; Sec. 3.2's largest
single-GPU size class) -- with one block product G X and one transpose block product G^T Y
on 2510 FP32 columns each (the RSVD block k + p = 2500 + 10 of Alg. 2).  Metric: column
products per second (G and G^T columns), whole job.  The inputs (X 10 GB, Y 0.5 GB) exceed
the 126 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c4|c2] [--dtype f32|f64]
                  [--impl reference]

Beside the headline the line carries, for the same configuration: the FP64 (plain path)
rate on a smaller block, the relative 2-norm error of sampled FP32 and FP64 columns against
the FP64 oracle, the c2 configuration's rate (100 x 100 stations, 1260 columns), the
end-to-end rate through the C ABI's host-buffer call, the roofline of the dominant kernel
and the oracle's own rate on one host core and on all of them.

Under torchrun each rank runs its own block (weak scaling, no collective on the data path);
the timed region is bracketed by a barrier and synchronisation and the maximum over ranks is
reported.  --impl reference times the FP64 CPU oracle (numpy FFT route) on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOADS = {
    "c4": dict(block=2510, kind="gravity", inc=90.0, dec=0.0,
               text="c4 gravity: 250x200 stations, 250x200x20 cells of 50 m, m=50000, "
                    "n=1000000; G X and G^T Y on 2510 columns per step"),
    "c2": dict(block=1260, kind="gravity", inc=90.0, dec=0.0,
               text="c2 gravity: 100x100 stations, 110x110x10 cells of 50 m (5% padding), "
                    "m=10000, n=121000; G X and G^T Y on 1260 columns per step"),
}
METRIC = "G/G^T column products per second"

# DRAM traffic per launch of the dominant kernel from an ncu capture, keyed by the hash of
# the kernel sources at capture time (null once the kernels change): the bytes of one
# captured launch scaled to the benchmark's launch by its columns.
# c4, FP32, one 64-column launch each: cols_fwd 590.9 MB (DRAM read 583.5 + write 7.4), cols_adj 535.6 MB
# (read 55.0 + write 480.6).
NCU_TRAFFIC = {
    ("cols_fwd", "c4", "f32"): {"hash": "257b18585c537d5d", "bytes_per_launch": 590.9e6, "columns": 64},
    ("cols_adj", "c4", "f32"): {"hash": "257b18585c537d5d", "bytes_per_launch": 535.6e6, "columns": 64},
}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("tf_ct_kernels.cuh", "tf_fft_ct.cuh", "tf_fft.cuh", "tf_check.cuh", "tf_bulk.cuh", "tf_tmem.cuh"):
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
    rows share one complex transform.  Bytes: FP32 values moved once."""
    n1, n2 = g.n1min, g.n2min
    nh = n1 // 2 + 1
    rows_m = g.nz * g.ny
    return {
        "rows_r2c_model": (rows_m / 2 * fft_flops(n1), 4 * g.n + 8 * rows_m * nh),
        "cols_fwd": ((g.nz + 1) * nh * fft_flops(n2) + 8 * g.nz * nh * n2,
                     8 * rows_m * nh + 8 * g.sy * nh),
        "rows_c2r_data": (g.sy / 2 * fft_flops(n1), 8 * g.sy * nh + 4 * g.m),
        "rows_r2c_data": (g.sy / 2 * fft_flops(n1), 4 * g.m + 8 * g.sy * nh),
        "cols_adj": ((g.nz + 1) * nh * fft_flops(n2) + 6 * g.nz * nh * n2,
                     8 * g.sy * nh + 8 * rows_m * nh),
        "rows_c2r_model": (rows_m / 2 * fft_flops(n1), 8 * rows_m * nh + 4 * g.n),
    }


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
                 "--format=csv,noheader,nounits", "-lms", "100"],
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


# ---------------------------------------------------------------------- CPU oracle legs

def _oracle_columns(args):
    """Worker of the CPU baseline: the oracle's FFT-route products (FP64, as it stands) on
    seeded columns of the workload, for about `seconds`; returns (products, seconds)."""
    cfg, seconds, seed = args
    from oracle import operator as oop
    g = synth.config_grid(cfg)
    w = WORKLOADS[cfg]
    T = oop.layer_tables(g, w["kind"], w["inc"], w["dec"])
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(g.n)
    y = rng.standard_normal(g.m)
    t0 = time.perf_counter()
    done = 0
    while True:
        oop.fft_matvec(g, T, x)
        oop.fft_rmatvec(g, T, y)
        done += 2
        if time.perf_counter() - t0 > seconds:
            break
    return done, time.perf_counter() - t0


def cpu_oracle_rates(cfg: str, seconds: float):
    """The oracle on one host core, then one process per host core (spawned, so that no
    CUDA state is inherited), each over the same bounded sample length."""
    one, dt1 = _oracle_columns((cfg, seconds, 1))
    cores = os.cpu_count() or 1
    env_threads = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            t0 = time.perf_counter()
            res = pool.map(_oracle_columns, [(cfg, seconds, 100 + k) for k in range(cores)])
            wall = time.perf_counter() - t0
    finally:
        if env_threads is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = env_threads
    done = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return {"one": (one / dt1, one, dt1), "all": (done / busy, done, busy, cores, wall)}


def run_reference(args):
    """The oracle as it stands (FP64 numpy FFT route, one host core) on a bounded sample
    of the workload: per step 2 G and 2 G^T columns."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import operator as oop
    cfg = args.config
    w = WORKLOADS[cfg]
    g = synth.config_grid(cfg)
    T = oop.layer_tables(g, w["kind"], w["inc"], w["dec"])
    rng = np.random.default_rng(123)
    per_step = 2
    X = rng.standard_normal((per_step, g.n))
    Y = rng.standard_normal((per_step, g.m))

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
    sample = f"{per_step} G and {per_step} G^T columns per step (of {w['block']}), FP64, 1 core"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "products/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["text"], "block_columns": per_step, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "products/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------- GPU legs

def _timed_steps(torch, op, X, Y, D, XT, steps, warmup, stream):
    def step():
        op.matmat(X, out=D)
        op.rmatmat(Y, out=XT)

    for _ in range(max(warmup, 1)):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _rel_err_sampled(torch, op, g, T, X, Y, D, XT, cols):
    """Relative 2-norm error of sampled columns of G X and G^T Y against the oracle's FP64
    FFT route applied to the same (device-precision) input columns."""
    from oracle import operator as oop
    worst = 0.0
    for b in cols:
        x = X[b].double().cpu().numpy()
        y = Y[b].double().cpu().numpy()
        ref_d = oop.fft_matvec(g, T, x)
        ref_x = oop.fft_rmatvec(g, T, y)
        e1 = np.linalg.norm(D[b].double().cpu().numpy() - ref_d) / np.linalg.norm(ref_d)
        e2 = np.linalg.norm(XT[b].double().cpu().numpy() - ref_x) / np.linalg.norm(ref_x)
        worst = max(worst, e1, e2)
    return worst


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--config", default="c4", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline (no FP64/c2/error/CPU legs): for profiling runs")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="column chunks of the host-buffer call (tf_products_host)")
    ap.add_argument("--columns", type=int, default=0,
                    help="columns per block (default: the workload's RSVD block); smaller "
                         "blocks serve profiling captures")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
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

    cfg = args.config
    w = WORKLOADS[cfg]
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    esz = 4 if dt == torch.float32 else 8
    g = synth.config_grid(cfg)
    op = Operator(g, w["kind"], w["inc"], w["dec"], dtype=dt)
    dev = torch.device("cuda", local)
    B = args.columns or w["block"]
    gen = torch.Generator(device=dev).manual_seed(123 + rank)
    X = torch.randn((B, g.n), generator=gen, device=dev, dtype=dt)
    Y = torch.randn((B, g.m), generator=gen, device=dev, dtype=dt)
    D = torch.empty((B, g.m), dtype=dt, device=dev)
    XT = torch.empty((B, g.n), dtype=dt, device=dev)
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
    products = 2 * B * args.steps * world
    value = products / (ms / 1e3)

    # end to end through the C ABI's host-buffer call (tf_products_host), pinned host blocks,
    # every step's copies in and out inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        Xh = torch.empty((B, g.n), dtype=dt, pin_memory=True)
        Yh = torch.empty((B, g.m), dtype=dt, pin_memory=True)
        Xh.copy_(X)
        Yh.copy_(Y)
        Dh = torch.empty((B, g.m), dtype=dt, pin_memory=True)
        XTh = torch.empty((B, g.n), dtype=dt, pin_memory=True)
        for _ in range(2):   # the first calls pay one-time costs (staging allocation, mappings)
            op.products_host(Xh, Yh, Dh, XTh, chunks=args.e2e_chunks)
            torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        step_ms = []
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            op.products_host(Xh, Yh, Dh, XTh, chunks=args.e2e_chunks)
            torch.cuda.synchronize()
            step_ms.append(round(1e3 * (time.perf_counter() - t1), 2))
        e2e_s = time.perf_counter() - t0
        barrier()
        e2e_s = max_over_ranks(e2e_s, dev)
        e2e = {"value": 2 * B * args.e2e_steps * world / e2e_s, "unit": "products/s",
               "h2d_bytes_per_step": (g.n + g.m) * B * esz,
               "d2h_bytes_per_step": (g.m + g.n) * B * esz,
               "call": "tf_products_host (C ABI), pinned host blocks, "
                       f"{args.e2e_chunks} chunks per step", "step_ms": step_ms}
        del Xh, Yh, Dh, XTh

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
    tr = NCU_TRAFFIC.get((top, cfg, args.dtype))
    ok = tr and tr["hash"] == kernel_hash() and B == w["block"]
    roof["traffic"] = tr["bytes_per_launch"] * per_launch_cols / tr["columns"] if ok else None
    roof["kernel"] = top
    roof["launch_ms"] = avg_s * 1e3
    roof["columns_per_launch"] = per_launch_cols
    total_stage = max(sum(v[0] for v in prof.values()), 1e-30)
    stage_share = {s: prof[s][0] / total_stage for s in STAGES}
    step_flops = sum(model[s][0] for s in STAGES) * B
    hbm_alg = (esz * g.n + esz * g.m) * 2 * B * args.steps / (ms / 1e3) / 1e9
    gpu_launches = int(sum(v[1] for v in prof.values()))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "products/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": w["text"], "block_columns": B, "fft": [op.n1, op.n2],
                   "tuning": list(op.tuning()),
                   "l2": (f"inputs (X {g.n * B * esz / 1e6:.0f} MB, Y {g.m * B * esz / 1e6:.0f} MB) "
                          + ("exceed L2; no flush" if g.n * B * esz > 129e6 else "fit in L2"))},
        "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roof,
        "step_alu_frac": step_flops * args.steps / (ms / 1e3) / 1e12 / measured,
        "hbm_algorithmic_gbs": hbm_alg, "stage_share": stage_share, "clocks": clk,
    }

    if world == 1 and not args.no_extras:
        from oracle import operator as oop
        T = oop.layer_tables(g, w["kind"], w["inc"], w["dec"])
        extras = {}
        # relative error of the timed block's sampled columns against the FP64 oracle
        extras["rel_err_vs_oracle"] = {
            args.dtype: _rel_err_sampled(torch, op, g, T, X, Y, D, XT, (0, B // 2, B - 1))}
        del X, Y, D, XT
        op.close()
        torch.cuda.empty_cache()
        # the other precision on a smaller block (FP64 is the plain path)
        other = torch.float64 if dt == torch.float32 else torch.float32
        oname = "f64" if other == torch.float64 else "f32"
        Bo = min(B, 256)
        op2 = Operator(g, w["kind"], w["inc"], w["dec"], dtype=other)
        gen = torch.Generator(device=dev).manual_seed(7)
        X2 = torch.randn((Bo, g.n), generator=gen, device=dev, dtype=other)
        Y2 = torch.randn((Bo, g.m), generator=gen, device=dev, dtype=other)
        D2 = torch.empty((Bo, g.m), dtype=other, device=dev)
        XT2 = torch.empty((Bo, g.n), dtype=other, device=dev)
        ms2 = _timed_steps(torch, op2, X2, Y2, D2, XT2, 3, 1, stream)
        extras[oname] = {"value": 2 * Bo * 3 / (ms2 / 1e3), "unit": "products/s",
                         "block_columns": Bo, "ms_per_step": ms2 / 3}
        extras["rel_err_vs_oracle"][oname] = _rel_err_sampled(
            torch, op2, g, T, X2, Y2, D2, XT2, (0, Bo - 1))
        del X2, Y2, D2, XT2
        op2.close()
        torch.cuda.empty_cache()
        # the c2 configuration (the paper's 100 x 100 station class, 1260-column RSVD block)
        if cfg != "c2":
            g2 = synth.config_grid("c2")
            w2 = WORKLOADS["c2"]
            op3 = Operator(g2, w2["kind"], w2["inc"], w2["dec"], dtype=dt)
            B3 = w2["block"]
            gen = torch.Generator(device=dev).manual_seed(11)
            X3 = torch.randn((B3, g2.n), generator=gen, device=dev, dtype=dt)
            Y3 = torch.randn((B3, g2.m), generator=gen, device=dev, dtype=dt)
            D3 = torch.empty((B3, g2.m), dtype=dt, device=dev)
            XT3 = torch.empty((B3, g2.n), dtype=dt, device=dev)
            ms3 = _timed_steps(torch, op3, X3, Y3, D3, XT3, 20, 3, stream)
            extras["c2"] = {"value": 2 * B3 * 20 / (ms3 / 1e3), "unit": "products/s",
                            "block_columns": B3, "ms_per_step": ms3 / 20, "dtype": args.dtype}
            del X3, Y3, D3, XT3
            op3.close()
        line["extras"] = extras
        rates = cpu_oracle_rates(cfg, args.cpu_seconds)
        r1, n1, s1 = rates["one"]
        ra, na, sa, cores, wall = rates["all"]
        line["cpu_baseline"] = {
            "value": r1, "unit": "products/s", "cores": 1, "kind": "oracle",
            "sample": f"{n1} FP64 column products (numpy FFT route, G and G^T alternating) in "
                      f"{s1:.1f} s on one core; host has {os.cpu_count()} cores"}
        line["cpu_baseline_all_cores"] = {
            "value": ra, "unit": "products/s", "cores": cores, "kind": "oracle",
            "sample": f"{na} FP64 column products over {cores} spawned processes, one per core, "
                      f"each for about {args.cpu_seconds:.0f} s (pool wall time {wall:.1f} s)"}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
