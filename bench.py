"""Throughput benchmark of the fused GB300 coupled-LB step (arXiv 2210.07501).

Workload: the bandwidth channel of 8192 x 2048 nodes (16.8M), bottom layer b = 1365
(a/b = 0.5), four heating periods, W = 5, sigma = 1e-3 - 1e-4 (T - 1)^2, D2Q9 flow +
D2Q5 phase field + D2Q5 energy, populations stored as FP32 deviations, FP32 arithmetic.
Synthetic: the initial state is the paper's rest state (tanh interface, T = T_ref).

One step = one pass of the whole hot path: the fused pull-stream-collide kernel for all
three lattices, plus the residual/mass reductions every 100 steps.  The working set
(2.7 GB) is 20x the L2, so no flush is needed between steps.

Prints one JSON line.  `--impl reference` times the CPU oracle instead (the only
reference this method has), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lbm_workloads as WL  # noqa: E402

METRIC = "MLUPS (coupled 3-lattice step) & HBM GB/s vs peak; sweep time-to-steady, warm vs cold"
WORKLOAD = "srf-channel-8192x2048"
PRECISION = "fp32"   # storage of the benchmark line (--precision changes it)
KERNEL_TYPES = {"fp32": "float,float", "fp16": "float,__half", "fp64": "double,double"}
CHECK_INTERVAL = 100


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws):
    """Replicas only: a process group just for the barrier and the max over ranks."""
    if ws <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend="gloo")
    return dist


def max_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def ncu_traffic():
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary, or None
    when the kernel source has changed since those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_kernel_fp32_8192x2048.json")
    csrc = os.path.join(ROOT, "paper_2210_07501_gb300", "csrc")
    try:
        with open(path) as f:
            d = json.load(f)
        h = hashlib.sha256(open(os.path.join(csrc, "lbm_step.cu"), "rb").read() +
                           open(os.path.join(csrc, "lbm_device.cuh"), "rb").read()).hexdigest()[:16]
        return d["dram_bytes_per_launch_full_size"] if d.get("source_sha256_16") == h else None
    except Exception:
        return None


def run_cpu_sample(budget_s: float, threads: int, nx=8192, ny=2048):
    """The oracle, as it stands, on the host cores: full-width channel of the benchmark
    workload; the number of rows is picked so that timed steps take about budget_s."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(threads) if threads > 0 else oracle.set_threads(0)
    # calibrate on a small strip of the same channel
    w = WL.workload(WORKLOAD, ny=64, b=43.0)
    o = oracle.Oracle(w["domain"], w["params"])
    o.step(1)
    t = time.perf_counter()
    o.step(1)
    rate = nx * 64 / max(time.perf_counter() - t, 1e-6)
    o.close()
    rows = int(min(ny, max(64, budget_s * rate / nx / 3.0)))
    w = WL.workload(WORKLOAD, ny=rows, b=round(rows / 1.5))
    o = oracle.Oracle(w["domain"], w["params"])
    o.step(1)
    steps = 3
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    o.close()
    mlups = nx * rows * steps / dt / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} timed steps of a {nx}x{rows} strip of the {WORKLOAD} channel "
                      f"(a/b = 0.5), FP64, after 1 warm-up step; {dt:.1f} s"}


def bench_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    nx = 8192
    w = WL.workload(WORKLOAD, ny=32, b=21.0)
    o = oracle.Oracle(w["domain"], w["params"])
    o.step(1)
    t = time.perf_counter()
    o.step(1)
    rate = nx * 32 / max(time.perf_counter() - t, 1e-6)
    o.close()
    budget = 90.0
    rows = int(max(3, min(2048, budget * rate / ((args.steps + args.warmup) * nx))))
    w = WL.workload(WORKLOAD, ny=rows, b=max(1.0, round(rows / 1.5)))
    o = oracle.Oracle(w["domain"], w["params"])
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    o.close()
    sites = nx * rows
    value = sites * args.steps / dt / 1e6
    sample = (f"each step: one oracle step of a {nx}x{rows} strip of the {WORKLOAD} channel (a/b = 0.5), "
              f"FP64 on {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": nx, "ny": rows, "storage": "fp64", "sampled": True},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def end_to_end(g, args, dist, ws, N, nx, ny):
    """Same metric through the C ABI with host buffers: the state goes up from pinned FP64
    host arrays (lbm_set_state), K steps run, the fields come back into pinned host arrays
    (lbm_fields); all inside the timed region."""
    import ctypes

    import torch
    st = g.lbm_get_state()
    pinned = {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True) for k, v in st.items()}
    for k in st:
        pinned[k].numpy()[...] = st[k]
    host = {k: pinned[k].numpy() for k in st}
    outs = {k: torch.empty((ny, nx), dtype=torch.float64, pin_memory=True) for k in ("phi", "u", "v", "T", "dp")}
    out_np = {k: t.numpy() for k, t in outs.items()}
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    g.lbm_set_state(host)                 # allocates the staging buffer outside the timed region
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    g.lbm_set_state(host)
    g.lbm_step(args.steps)
    rc = g._lib.lbm_fields(g._h, *[ptr(out_np[k]) for k in ("phi", "u", "v", "T", "dp")])
    t1 = time.perf_counter()
    if rc != 0:
        raise RuntimeError("lbm_fields failed")
    e2e_s = max_over_ranks(dist, t1 - t0)
    h2d = sum(a.nbytes for a in host.values())
    d2h = sum(a.nbytes for a in out_np.values())
    return {"value": ws * N * args.steps / e2e_s / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps}


def bench_gpu(args):
    import torch

    import paper_2210_07501_gb300 as pkg
    ws, rank, local = dist_env()
    dist = init_dist(ws)
    torch.cuda.set_device(local)
    pkg.build()
    pkg.load()
    w = WL.workload(WORKLOAD)
    if args.ny:   # a shorter channel of the same workload, for profiler captures
        w = WL.workload(WORKLOAD, ny=args.ny, b=round(args.ny / 1.5))
    nx, ny = w["domain"]["nx"], w["domain"]["ny"]
    N = nx * ny
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = pkg.Lbm(w["domain"], w["params"], precision=args.precision, stream=stream)
        g.lbm_set_check_interval(CHECK_INTERVAL)
        bpn = g.lbm_bytes_per_node()
        if args.segment:
            g.lbm_set_segment(args.segment)
            seg_rows = args.segment
        else:
            seg_rows = g.lbm_autotune(10)    # launch shape; leaves the state untouched
        # ---- device-resident throughput ----
        g.lbm_step(args.warmup)
        torch.cuda.synchronize()
        barrier(dist)
        torch.cuda.synchronize()
        l0 = g.lbm_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            g.lbm_step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        barrier(dist)
        launches = g.lbm_launch_count() - l0
        checks = sum(1 for s in range(args.warmup + 1, args.warmup + args.steps + 1) if s % CHECK_INTERVAL == 0)
        gpu_launches = launches + 2 * checks
        diag = g.lbm_diag(raise_unstable=False)
        ms_max = max_over_ranks(dist, ms)
        value = ws * N * args.steps / (ms_max * 1e-3) / 1e6
        # ---- end to end through the C ABI with host buffers ----
        e2e = None if args.no_e2e else end_to_end(g, args, dist, ws, N, nx, ny)
        g.close()
    clocks = clk.summary()
    peak, peak_kind = measured_peaks()
    ms_step = ms / args.steps
    achieved = N * bpn / (ms_step * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "b": w["domain"]["b"], "W": w["domain"]["W"],
                   "lattices": "D2Q9 flow + D2Q5 phase field + D2Q5 energy", "storage": args.precision,
                   "check_interval": CHECK_INTERVAL, "l2": "working set 2.7 GB > L2 (no flush needed)",
                   "segment_rows": seg_rows,
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": ncu_traffic() if args.precision == PRECISION else None,
                     "bytes_per_node": bpn, "peak_source": peak_kind,
                     "kernel": f"lbm::march_kernel<{KERNEL_TYPES[args.precision]},5,5,128> "
                               "(+ reductions every 100 steps in the region)"},
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "diag": {"mass": diag["mass"], "residual": diag["residual"], "unstable": diag["unstable"]},
    }
    if args.ny:
        line["config"]["reduced_rows_for_profiling"] = args.ny
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_sample(args.cpu_budget, 0)
        one = run_cpu_sample(args.cpu_budget / 3.0, 1)      # the same oracle on one host thread
        line["cpu_baseline"]["single_thread"] = {"value": one["value"], "unit": one["unit"], "sample": one["sample"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def bench_sweep(args):
    """Batched uneven sweep against the plain per-case solver: wall time to steady state
    (residual <= tol) for the first `args.sweep` channels of the seeded 96-channel sweep."""
    import torch

    import paper_2210_07501_gb300 as pkg
    pkg.build()
    pkg.load()
    cases = WL.sweep_cases(96, seed=0)[:args.sweep]
    K = args.sweep_k
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = pkg.LbmBatch(cases, precision="fp32")
    b.lbm_batch_set_check_interval(K)
    rows = b.lbm_batch_autotune(5)
    steps_b, conv_b = b.lbm_batch_run_to_steady(args.sweep_tol, args.sweep_max)
    t_batch = time.perf_counter() - t0
    size = b.lbm_batch_size()
    b.close()
    t0 = time.perf_counter()
    steps_s, conv_s = [], []
    for w in cases:
        g = pkg.Lbm(w["domain"], w["params"], precision="fp32")
        g.lbm_set_check_interval(K)
        g.lbm_autotune(3)
        ok, n = g.lbm_run_to_steady(args.sweep_tol, args.sweep_max)
        steps_s.append(n)
        conv_s.append(ok)
        g.close()
    t_single = time.perf_counter() - t0
    sites = [w["domain"]["nx"] * w["domain"]["ny"] for w in cases]
    lu = sum(s * n for s, n in zip(sites, steps_b))
    line = {"sweep": {
        "cases": len(cases), "generator": "seeded sweep_cases(96, seed=0), first cases", "precision": "fp32",
        "tol": args.sweep_tol, "max_steps": args.sweep_max, "check_interval": K,
        "batched_s": t_batch, "per_case_s": t_single, "speedup": t_single / t_batch,
        "converged_batched": int(sum(conv_b)), "converged_per_case": int(sum(conv_s)),
        "same_steps": steps_b == steps_s, "batched_mlups": lu / t_batch / 1e6,
        "batch_ctas": size["ctas"], "segment_rows": rows,
        "steps": steps_b, "sites_total": sum(sites)}}
    print(json.dumps(line), flush=True)
    return 0


def bench_trends(args):
    """The parametric study of Sec. 6 as one batched FP64 sweep: U_max on the interface
    against k~ and mu~ for a/b = 1/3, 1, 3 and against M2 (the comparison with the
    closed form of Sec. 3 is made in tests/test_gpu_trends.py)."""
    import paper_2210_07501_gb300 as pkg
    from paper_2210_07501_gb300 import trends as T
    pkg.build()
    pkg.load()
    cl = (T.cases("cond_ratio", (0.25, 0.5, 1.0, 2.0, 4.0)) + T.cases("visc_ratio", (0.25, 0.5, 2.0, 4.0)) +
          T.cases("M2", (2.5e-2, 1e-1), ab_values=(1.0,)))
    res, seconds = T.run(cl, tol=args.sweep_tol if args.sweep_tol < 1e-5 else 1e-6, max_steps=args.sweep_max)
    sites = sum(c["domain"]["nx"] * c["domain"]["ny"] for c in cl)
    lu = sum(c["domain"]["nx"] * c["domain"]["ny"] * r["steps"] for c, r in zip(cl, res))
    line = {"trends": {"cases": len(cl), "precision": "fp64", "seconds": seconds, "sites_total": sites,
                       "batched_mlups": lu / seconds / 1e6,
                       "rows": [{"name": r["name"], "steps": r["steps"], "converged": r["converged"],
                                 "U_lb": r["U_lb"]} for r in res]}}
    print(json.dumps(line), flush=True)
    return 0


def bench_warmstart(args):
    """Learned warm start: surrogate trained on solver-generated steady channels (256 x 64),
    then warm vs cold starts on held-out seeds."""
    import paper_2210_07501_gb300 as pkg
    from paper_2210_07501_gb300 import warmstart
    pkg.build()
    pkg.load()
    n_train, n_test = args.warmstart
    train = WL.surrogate_cases(n_train, seed=1000)
    test = WL.surrogate_cases(n_test, seed=2000)
    r = warmstart.experiment(train, test, tol=args.warm_tol, max_steps=args.warm_max, K=args.warm_k,
                             train_tol=args.train_tol, train_max_steps=args.train_max, iters=args.train_iters,
                             batch=16, lr=1e-3, seed=0, plain_cases=args.warm_plain)
    print(json.dumps({"warmstart": r}), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--ny", type=int, default=0, help="rows of a shorter channel (profiling); 0 = full")
    ap.add_argument("--segment", type=int, default=0, help="rows per CTA segment; 0 = autotune")
    ap.add_argument("--precision", choices=["fp32", "fp16", "fp64"], default=PRECISION,
                    help="storage precision (fp16: FP32 arithmetic; fp64: FP64 throughout)")
    ap.add_argument("--sweep", type=int, default=0, help="run the batched-sweep comparison on N channels")
    ap.add_argument("--trends", action="store_true", help="run the Sec. 6 parametric study (U_max trends)")
    ap.add_argument("--sweep-tol", type=float, default=1e-5)
    ap.add_argument("--sweep-max", type=int, default=60000)
    ap.add_argument("--sweep-k", type=int, default=100, help="sweep: steps between residual checks (even)")
    ap.add_argument("--warmstart", type=int, nargs=2, default=None, metavar=("TRAIN", "TEST"),
                    help="learned warm start: train on TRAIN channels, compare on TEST channels")
    ap.add_argument("--train-iters", type=int, default=3000)
    ap.add_argument("--warm-tol", type=float, default=1e-8, help="warm start: residual of the held-out runs")
    ap.add_argument("--warm-k", type=int, default=1000, help="warm start: steps between residual checks")
    ap.add_argument("--warm-max", type=int, default=3000000)
    ap.add_argument("--warm-plain", type=int, default=0, help="warm start: held-out cases also run one by one")
    ap.add_argument("--train-tol", type=float, default=1e-6, help="warm start: residual of the training runs")
    ap.add_argument("--train-max", type=int, default=400000)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return bench_reference(args)
    if args.sweep:
        return bench_sweep(args)
    if args.warmstart:
        return bench_warmstart(args)
    if args.trends:
        return bench_trends(args)
    return bench_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
