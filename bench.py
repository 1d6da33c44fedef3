"""Benchmark of the PDMCF hot path on GB300: PDHG iterations per second.

Default workload (one GPU): the large single solve, n = 10^4 nodes, m = 10^5 edges (directed
ring plus 9 random out-edges per node), capacities lognormal(0, 0.5), power utility
w s^0.5 with w ~ U[0.5, 1.5]; F is 10^4 x 10^5 (10^9 variables) in FP32. A step is one PDHG
iteration (edge phase, node phase, scalar tail; every k_check-th iteration also the
residual check), launched through the C ABI on torch's current stream.

Printed JSON line (rank 0):
  value     iterations/s of the whole job (sum over ranks / max time), inputs resident in HBM
  e2e       the same metric through the public API with host buffers: problem creation
            (host -> device copies), the solve, and the read-back of T inside the timed region
  roofline  the dominant kernel: algorithmic bytes per launch / its mean CUDA-event duration,
            against the measured HBM copy bandwidth
  cpu_baseline  the FP64 CPU oracle timed on a bounded sample (the same recipe at n = 1000),
            scaled to this workload by the ratio of n m
  --impl reference  times that oracle alone as the reference arm.
"""
from __future__ import annotations

import os

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2501_17996_gb300 import instances as I  # noqa: E402

METRIC = "PDHG iters/s, HBM GB/s vs peak; served p50/p99 solve latency @1e-4 KKT"

WORKLOADS = {
    "large": dict(factory=lambda seed: I.large(seed), sample=lambda seed: I.large_slice(seed),
                  desc="n=10000, m=100000 (ring + 9 random out-edges per node), "
                       "c~lognormal(0,0.5), u = w s^0.5, w~U[0.5,1.5]"),
    # profiling case: the large per-edge vector length (n = 10^4, same kernel shape) with
    # out-degree 2, so one capture holds ~4 GB on the device
    "prof": dict(factory=lambda seed: I.ring_random_instance(10000, 2, seed, "lognormal", "pow",
                                                             gamma=0.5, name="prof"),
                 sample=lambda seed: I.large_slice(seed),
                 desc="n=10000, m=20000 (ring + 1 random out-edge per node), large recipe"),
    "mid": dict(factory=lambda seed: I.mid(seed), sample=lambda seed: I.mid(seed),
                desc="n=100, m=1000 (ring + 9 random out-edges per node), c~U[1,10], "
                     "u = w log s, w~U[0.5,1.5]"),
}


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2501_17996_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cuh", ".cu", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def algorithmic_bytes(n: int, m: int, s_f: int, s_p: int = 4) -> dict:
    """Bytes each kernel must move per launch (each array touched once):
    edge:   read F^{k-1/2}, write F^{k+1/2} (2 s_F n m), read Y once (s_P n^2), 16 m of
            incidence, capacity and mu;
    node:   read F^{k+1/2} once (s_F n m), read Y, W, P and write Y, P (5 s_P n^2), 4(m+2n);
    check:  read F^{k-1/2} once (s_F n m), read Y, U', Y^ once (3 s_P n^2), 12 m;
    iteration (edge + node): 3 s_F n m + 6 s_P n^2 + ~20 m; the method's floor of
    2 s_F n m + 3 s_P n^2 is reported beside it."""
    nm, n2 = float(n) * m, float(n) * n
    return {
        "edge": 2 * s_f * nm + s_p * n2 + 16 * m,
        "node": s_f * nm + 5 * s_p * n2 + 4 * (m + 2 * n),
        "check": s_f * nm + 3 * s_p * n2 + 12 * m,
        "scalar": 0.0,
        "iteration_floor": 2 * s_f * nm + 3 * s_p * n2,
    }


# ------------------------------------------------------------------ clocks sampler

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.device), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm_, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm_)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle timing

def oracle_iters_per_s(sample, k_check: int, steps: int, warmup: int):
    """Time `steps` oracle iterations on the sample instance (cold start each call):
    t(warmup + steps) - t(warmup) so start-up work cancels."""
    from oracle import pdmcf as O

    def run(k):
        t0 = time.perf_counter()
        O.pdmcf(sample.n, sample.tail, sample.head, sample.cap, sample.kind, sample.w,
                sample.gamma, stop_mode="none", max_iters=k, k_check=k_check)
        return time.perf_counter() - t0

    t_w = run(warmup) if warmup > 0 else 0.0
    t_all = run(warmup + steps)
    dt = max(t_all - t_w, 1e-9)
    return steps / dt, dt


def cpu_baseline(wl, inst, seed, k_check, steps=6, warmup=1):
    sample = wl["sample"](seed)
    ips, dt = oracle_iters_per_s(sample, k_check, steps, warmup)
    scale = (sample.n * sample.m) / float(inst.n * inst.m)
    return {
        "value": ips * scale,
        "unit": "iters/s",
        "cores": 1,
        "kind": "oracle",
        "sample": (f"{steps} FP64 oracle iterations (single-threaded numpy/scipy) on the same "
                   f"recipe at n={sample.n}, m={sample.m} ({dt:.1f} s), scaled by "
                   f"n m ratio {scale:.3g} to the full workload"),
    }


# ------------------------------------------------------------------ arms

def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    inst_n, inst_m = {"large": (10000, 100000), "prof": (10000, 20000), "mid": (100, 1000)}[args.workload]
    sample = wl["sample"](args.seed)
    if args.workload == "large" and args.steps + args.warmup > 60:
        sample = I.large(args.seed, n=500)
    ips, dt = oracle_iters_per_s(sample, args.k_check, args.steps, args.warmup)
    scale = (sample.n * sample.m) / float(inst_n * inst_m)
    value = ips * scale
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "n": inst_n, "m": inst_m},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle",
                         "sample": (f"each step one FP64 oracle iteration on the same recipe at "
                                    f"n={sample.n}, m={sample.m}; {args.steps} steps took "
                                    f"{dt:.1f} s; scaled by n m ratio {scale:.3g}")},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2501_17996_gb300 import binding as B

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    wl = WORKLOADS[args.workload]
    seed = args.seed + rank
    inst = wl["factory"](seed)
    n, m = inst.n, inst.m
    prec = args.precision
    s_f = {"fp32": 4, "bf16": 2, "fp64": 8}[prec]
    s_p = 8 if prec == "fp64" else 4
    common = dict(precision=prec, device=local_rank, k_check=args.k_check,
                  cuda_stream=stream.cuda_stream, stop_mode="none")

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- device-resident timed region
    prob = B.Problem(inst)
    prob.solve(want_T=False, max_iters=max(args.warmup, 1), **common)     # allocate, upload, warm
    torch.cuda.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        res, times = prob.solve_timed(max_iters=args.steps, warm_start=1, **common)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * args.steps / (ms_max / 1e3)
    launches = sum(v[1] for k, v in times.items() if k != "ms_total")

    # ---- roofline of the dominant kernel
    alg = algorithmic_bytes(n, m, s_f, s_p)
    dom = max(("edge", "node", "check"), key=lambda k: times[k][0])
    dom_ms = times[dom][0] / max(times[dom][1], 1)
    peak, peak_kind = peaks()
    achieved = alg[dom] / (dom_ms / 1e3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", f"{dom}_kernel_{args.workload}_{prec}.json")
    if os.path.exists(prof):
        try:
            pj = json.load(open(prof))
            if pj.get("kernel_source_hash") == kernel_source_hash():
                traffic = pj.get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    iter_ms = ms / args.steps
    per_kernel = {k: {"ms_per_launch": (v[0] / v[1]) if v[1] else None, "launches": v[1],
                      "share": v[0] / max(times["ms_total"], 1e-9),
                      "alg_gbs": (alg[k] / (v[0] / v[1] / 1e3) / 1e9) if v[1] and alg[k] else None}
                  for k, v in times.items() if k != "ms_total"}
    prob.close()

    # ---- end to end through the public API with host buffers
    e2e_value = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        with B.Problem(inst) as p2:
            p2.solve(want_T=True, max_iters=args.steps, **common)
        t_e2e = time.perf_counter() - t0
        tt = torch.tensor([t_e2e], device="cuda")
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_value = world * args.steps / float(tt.item())
    ld = (n + 7) // 8 * 8
    h2d = (n * ld * s_p) + m * s_p + (3 * m + 2 * (n + 1)) * 4     # W, cap, incidence
    d2h = n * ld * s_p                                             # T

    # ---- time to tolerance (optional)
    ttt = None
    if args.ttt:
        with B.Problem(inst) as p3:
            t0 = time.perf_counter()
            r3 = p3.solve(want_T=False, max_iters=args.ttt_max_iters,
                          **{**common, "stop_mode": "kkt"}, eps=args.ttt_eps, raise_on_error=False)
            ttt = {"seconds": time.perf_counter() - t0, "iters": r3["iters"],
                   "rel_kkt": r3["rel_kkt"], "eps": args.ttt_eps, "status": r3["rc"]}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec != "fp64" else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "n": n, "m": m,
                   "precision": prec, "storage_F": {"fp32": "f32", "bf16": "bf16", "fp64": "f64"}[prec],
                   "k_check": args.k_check, "seed": args.seed,
                   "l2": "inputs larger than L2 (F alone is %.1f GB)" % (2 * s_f * n * m / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "alg_bytes_per_launch": alg[dom],
                     "ms_per_launch": dom_ms},
        "hbm": {"iteration_floor_gbs": alg["iteration_floor"] / (iter_ms / 1e3) / 1e9,
                "iteration_alg_gbs": (alg["edge"] + alg["node"]) / (iter_ms / 1e3) / 1e9,
                "peak_gbs": peak, "kernels": per_kernel},
        "e2e": {"value": e2e_value, "unit": "iters/s", "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps,
                "note": "problem creation + upload, %d iterations, T read-back" % args.steps},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if ttt:
        line["time_to_tolerance"] = ttt
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, inst, args.seed, args.k_check)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--k-check", dest="k_check", type=int, default=50)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ttt", action="store_true", help="also time a solve to --ttt-eps")
    ap.add_argument("--ttt-eps", dest="ttt_eps", type=float, default=1e-4)
    ap.add_argument("--ttt-max-iters", dest="ttt_max_iters", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", dest="no_cpu_baseline", action="store_true")
    ap.add_argument("--no-e2e", dest="no_e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
