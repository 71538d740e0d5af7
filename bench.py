"""Benchmark: time to an FP64-accurate A^{-1/p} on one GB300, through the library's C ABI.

One step = the whole hot path on the n = 4096, kappa = 1e3 SPD matrix (Q diag(lam) Q^T, lam log-uniform
in [1e-3, 1], seed 1) for every root index in --p: load A (checks, ||A||_1, ||A||_inf, C_0 of Eq. 3),
iterate Eq. 1 to the tolerance (precision ladder per --mode), the true residual ||I - C^p A||_F, and the
result copy. The value is milliseconds per step (lower is better). Inputs are resident in HBM before
the timed region; the working set (about 9 x 128 MiB per handle) exceeds the 129 MB L2.

`--impl reference` times the CPU oracle (numpy FP64) on the host cores instead, on a bounded sample
scaled to the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1703_02283_gb300 import workloads as W  # noqa: E402

METRIC = "time to FP64-accurate A^(-1/p) vs plain FP64 GPU; GEMM TFLOP/s, % of peak"
NOMINAL_BF16_TFLOPS = 2250.0
NOMINAL_FP64_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=W.SINGLE_CASE["n"])
    ap.add_argument("--lam-min", type=float, default=W.SINGLE_CASE["lam_min"])
    ap.add_argument("--seed", type=int, default=W.SINGLE_CASE["seed"])
    ap.add_argument("--p", default="2", help="comma-separated root indices solved in one step")
    ap.add_argument("--mode", default="fp64", choices=["fp64"], help="precision plan of the timed solve")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle timing

def oracle_sample(A: np.ndarray, p: int, iterations: int) -> tuple[float, str]:
    """Times the oracle's setup plus one and two updates and extrapolates to `iterations` updates."""
    from oracle import pthroot_oracle as O
    t0 = time.perf_counter()
    O.solve(A, p, tol=0.0, max_iter=1, stag_below=0.0)
    t1 = time.perf_counter()
    O.solve(A, p, tol=0.0, max_iter=2, stag_below=0.0)
    t2 = time.perf_counter()
    per_update = max((t2 - t1) - (t1 - t0), 1e-9)
    setup = max((t1 - t0) - per_update, 0.0)
    est = setup + per_update * iterations
    return est * 1e3, f"oracle setup + 1 and + 2 updates at n={A.shape[0]}, p={p}, extrapolated to {iterations} updates"


def predicted_iterations(case, p: int, tol: float) -> int:
    """Iterations the exact-arithmetic model (the oracle's scalar recurrence) needs to reach tol."""
    from oracle import pthroot_oracle as O
    s = O.norm_1(case.A) * O.norm_inf(case.A)
    r = O.scalar_residuals(case.lam, case.lam / s, p, 200)
    hit = np.nonzero(r <= max(tol, 1e-13))[0]
    return int(hit[0]) if len(hit) else 200


def run_reference(args, ps):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    case = W.spd_from_spectrum(args.n, args.lam_min, args.seed)
    total_ms, samples = [], []
    for _ in range(args.warmup + args.steps):
        ms = 0.0
        for p in ps:
            est, what = oracle_sample(case.A, p, predicted_iterations(case, p, args.tol))
            ms += est
            samples.append(what)
        total_ms.append(ms)
    timed = total_ms[args.warmup:]
    value = float(np.mean(timed))
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, ps),
            "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": samples[0] + " (each step, per p)"},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args, ps):
    return {"workload": f"SPD n={args.n}, kappa={1 / args.lam_min:g}, p={','.join(map(str, ps))}, "
                        f"Eq.3 C_0, tol {args.tol:g}", "n": args.n, "kappa": 1 / args.lam_min, "p": ps,
            "seed": args.seed, "mode": args.mode, "l2": "working set > 129 MB L2 (inputs larger than L2)"}


# ----------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    ps = [int(x) for x in args.p.split(",")]
    if args.impl == "reference":
        return run_reference(args, ps)

    import torch
    import torch.distributed as dist

    from paper_1703_02283_gb300 import pthroot as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream

    # Replicas: every rank solves its own matrix of the same recipe (seed offset by rank).
    case = W.spd_from_spectrum(args.n, args.lam_min, args.seed + 1000 * rank)
    A = torch.from_numpy(case.A).to(dev)
    C = torch.empty_like(A)
    prec = {"fp64": P.PR_FP64}[args.mode]
    handles = {}
    for p in ps:
        o = P.pr_default_options()
        handles[p] = P.pr_init(A, args.n, p, o, sptr)

    def step():
        info = {}
        for p, h in handles.items():
            P.pr_load(h, A)
            st, steps = P.pr_solve(h, prec, 0, prec, args.tol)
            res = P.pr_residual(h, prec)
            P.pr_result(h, C)
            info[p] = (st, steps, res)
        return info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    s0 = {p: P.pr_stats(h) for p, h in handles.items()}
    for h in handles.values():
        P.pr_set_timing(h, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        infos = [step() for _ in range(args.steps)]
        ev1.record(stream)
        barrier()
    for h in handles.values():
        P.pr_set_timing(h, False)
    ms = ev0.elapsed_time(ev1) / args.steps
    s1 = {p: P.pr_stats(h) for p, h in handles.items()}
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # Accuracy of the last step against the exact root (closed form, built on the host).
    from_closed = {}
    last = infos[-1]
    Cn = C.cpu().numpy()
    Zs = {p: (case.Q * case.lam ** (-1.0 / p)) @ case.Q.T for p in ps}
    for p, h in handles.items():
        P.pr_result(h, C)
        Cn = C.cpu().numpy()
        Z = Zs[p]
        from_closed[p] = float(np.linalg.norm(Cn - Z) / np.linalg.norm(Z))

    gemm_ms = sum(s1[p]["gemm_ms"] - s0[p]["gemm_ms"] for p in ps)
    gemm_fl = sum(s1[p]["gemm_flops_timed"] - s0[p]["gemm_flops_timed"] for p in ps)
    gemm_n = sum(s1[p]["gemms_timed"] - s0[p]["gemms_timed"] for p in ps)
    launches = sum(s1[p]["launches"] - s0[p]["launches"] for p in ps)
    peaks, peak_src = load_peaks()
    achieved = gemm_fl / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    if args.mode == "fp64":
        peak = peaks["bf16_tflops_sustained"] * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
        peak_note = f"{peak_src} bf16 sustained x nominal fp64/bf16 ratio ({NOMINAL_FP64_TFLOPS}/{NOMINAL_BF16_TFLOPS})"
        dtype = "f64"
    roofline = {"bound": "tensor", "kernel": "k_gemm_f64 (DMMA)", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": None,
                "peak_source": peak_note, "launches_timed": gemm_n,
                "flops_per_launch": gemm_fl / gemm_n if gemm_n else None,
                "avg_launch_ms": gemm_ms / gemm_n if gemm_n else None}

    # End to end through host buffers (pinned), copies inside the timed region.
    e2e = None
    if not args.no_e2e:
        Ah = torch.from_numpy(case.A).pin_memory()
        Ch = torch.empty_like(Ah).pin_memory()
        for _ in range(1):
            for p, h in handles.items():
                P.pr_load(h, Ah)
                P.pr_solve(h, prec, 0, prec, args.tol)
                P.pr_residual(h, prec)
                P.pr_result(h, Ch)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for p, h in handles.items():
                P.pr_load(h, Ah)
                P.pr_solve(h, prec, 0, prec, args.tol)
                P.pr_residual(h, prec)
                P.pr_result(h, Ch)
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        nbytes = args.n * args.n * 8 * len(ps)
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tot, what = 0.0, []
        for p in ps:
            est, w = oracle_sample(case.A, p, last[p][1])
            tot += est
            what.append(w)
        cpu = {"value": tot, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle", "sample": "; ".join(what)}

    for h in handles.values():
        P.pr_destroy(h)
    if rank == 0:
        line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config_dict(args, ps),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(),
                "solves": {str(p): {"status": P.STATUS_NAMES[last[p][0]], "iterations": last[p][1],
                                    "true_residual": last[p][2], "rel_error_vs_closed_form": from_closed[p]}
                           for p in ps}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
