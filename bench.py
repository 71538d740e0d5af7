"""Benchmark: time to an FP64-accurate A^{-1/p} on one GB300, through the library's C ABI.

Workload: the n = 4096, kappa = 1e3 SPD matrix (Q diag(lam) Q^T, lam log-uniform in [1e-3, 1], seed 1),
roots p = 1, 2, 3, 4, initial guess of Eq. 3, tolerance 1e-12 on the iteration's residual.

One step = the whole hot path for every p in --p: load A (checks, ||A||_1, ||A||_inf, C_0), iterate Eq. 1
to the tolerance or the precision floor, the true residual ||I - C^p A||_F and the result copy. The value is
milliseconds per step (lower is better) for --mode:
  fast   FP64-accurate products from exact FP16 digit slices (PR_EMU64) for every p; for p = 1, whose
         Newton-Schulz form corrects earlier errors, BF16 iterations first, then PR_EMU64 ones (default);
  emu64  PR_EMU64 for every iteration;
  fp64   native FP64 products (the plain FP64 GPU iteration).
Unless --no-compare, the plain FP64 GPU iteration is also run once per p in the same process and its time
and accuracy are reported beside the value. Inputs are resident in HBM before the timed region; the
working set (about 1.5 GiB per handle) exceeds the 129 MB L2.

`--impl reference` times the CPU oracle (numpy FP64) on the host cores instead, on a bounded sample scaled
to the same unit.
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
PREC_NAMES = {0: "fp64", 1: "emu64", 3: "bf16"}
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one symmetric product, by n. Taken before the kernel
# gained its split-tile variant; the unsplit code path that n = 4096 runs is unchanged (same registers and
# spills), but until it is captured again the roofline reports it as traffic_last_capture, not traffic.
EMU_TRAFFIC_BYTES = {4096: 2.371166e9 + 0.200156e9}


# ----------------------------------------------------------------------------- replicas (N > 1 under torchrun)
# Every workload runs one independent replica per rank (its own inputs, same recipe, seeds offset by rank):
# the problems do not share data, so no collective enters the data path. The ranks meet only at barriers
# around the timed region and in one MAX reduction of the timings; rank 0 prints.

def replica_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(seed: int, rank: int) -> int:
    return seed + 1000 * rank


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks of the default process group (x itself when there is none)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=W.SINGLE_CASE["n"])
    ap.add_argument("--lam-min", type=float, default=W.SINGLE_CASE["lam_min"])
    ap.add_argument("--seed", type=int, default=W.SINGLE_CASE["seed"])
    ap.add_argument("--p", default="1,2,3,4", help="comma-separated root indices solved in one step")
    ap.add_argument("--mode", default="fast", choices=["fast", "emu64", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--emu-slices", type=int, default=0, help="PR_EMU64 digit planes per operand (0: the default, 8)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "learned"],
                    help="single: the n=4096 matrix for every p; batched: 512 matrices, n in [64, 1024]")
    ap.add_argument("--count", type=int, default=512, help="batched: number of matrices")
    ap.add_argument("--learned-n", type=int, default=2048, help="learned: matrix order")
    ap.add_argument("--train-seqs", type=int, default=40, help="learned: training sequences (ids 0..)")
    ap.add_argument("--test-seqs", type=int, default=10, help="learned: held-out sequences (ids 40..)")
    ap.add_argument("--every", type=int, default=50, help="learned: sample every this many of 200 steps")
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
    return (setup + per_update * iterations) * 1e3, (f"n={A.shape[0]} p={p}: oracle setup + 1 and + 2 updates, "
                                                     f"extrapolated to {iterations} updates")


def predicted_iterations(case, p: int, tol: float) -> int:
    """Iterations the exact-arithmetic model (the oracle's scalar recurrence) needs to reach tol."""
    from oracle import pthroot_oracle as O
    s = O.norm_1(case.A) * O.norm_inf(case.A)
    r = O.scalar_residuals(case.lam, case.lam / s, p, 200)
    hit = np.nonzero(r <= max(tol, 1e-13))[0]
    return int(hit[0]) if len(hit) else 200


L2_BYTES = 129e6


def handle_bytes(n: int) -> float:
    """Device bytes a handle of order n works on: nine FP64 matrices, their BF16 copies and the digit
    planes (8 FP16 planes) of the six matrices the products slice."""
    ld = (n + 15) // 16 * 16
    return 9 * 8.0 * n * n + 9 * 2.0 * n * ld + 6 * 16.0 * n * ld


def l2_note(nbytes: float) -> str:
    side = "larger" if nbytes > L2_BYTES else "smaller"
    return f"inputs {side} than L2: working set {nbytes / 2**30:.3g} GiB vs 129 MB L2"


def config_dict(args, ps):
    return {"workload": f"SPD n={args.n} (Q diag(lam) Q^T), kappa={1 / args.lam_min:g}, p={','.join(map(str, ps))}, "
                        f"Eq.3 C_0, tol {args.tol:g}", "n": args.n, "kappa": 1 / args.lam_min, "p": ps,
            "seed": args.seed, "mode": args.mode,
            "l2": l2_note(handle_bytes(args.n)) + " per handle"}


def run_reference(args, ps):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    case = W.spd_from_spectrum(args.n, args.lam_min, args.seed)
    totals, samples = [], []
    for _ in range(args.warmup + args.steps):
        ms = 0.0
        for p in ps:
            est, what = oracle_sample(case.A, p, predicted_iterations(case, p, args.tol))
            ms += est
            samples.append(what)
        totals.append(ms)
    value = float(np.mean(totals[args.warmup:]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, ps),
            "cpu_baseline": {"value": value, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "; ".join(samples[:len(ps)]) + " (every step)"},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def batched_cases(count, rank=0):
    """The batch of one replica: rank 0 the benchmark's batch (specs seed 999, matrix seeds 1000 + i), other
    ranks the same recipe with their own seeds."""
    spec = W.batched_specs(count, seed=999 + rank)
    seeds = [int(x) + 100000 * rank for x in spec.seeds]
    cases = [W.spd_from_spectrum(int(spec.n[i]), float(spec.lam_min[i]), seeds[i]) for i in range(count)]
    return cases, [int(x) for x in spec.p]


def batch_bytes(count: int) -> float:
    """Device bytes of the packed batch: nine FP64 buffers and their digit planes, R rows x the largest order."""
    spec = W.batched_specs(count)
    R, K = int(spec.n.sum()), int(spec.n.max())
    ld = (K + 15) // 16 * 16
    return 9 * 8.0 * R * ld + 9 * 16.0 * R * ld


def batched_config(args):
    return {"workload": f"batched: {args.count} SPD matrices, n uniform in [64, 1024], kappa log-uniform in "
                        f"[10, 1e4], p in {{1, 2, 3}} (seeds 1000+i), Eq.3 C_0, tol {args.tol:g}",
            "count": args.count, "mode": "emu64",
            "step": "pr_batch_load of every matrix + pr_batch_solve (one graph launch) + every pr_batch_result",
            "l2": l2_note(batch_bytes(args.count)) + " (packed batch)"}


def oracle_batched_sample(cases, ps, its, k=3):
    """Oracle time on k matrices (setup + 1, 2 updates each), scaled to the batch by sum(n^3 iterations)."""
    rng = np.random.default_rng(1)
    idx = rng.choice(len(cases), k, replace=False)
    t = 0.0
    for i in idx:
        est, _ = oracle_sample(cases[i].A, ps[i], its[i])
        t += est
    work = lambda i: cases[i].n ** 3 * max(its[i], 1)  # noqa: E731
    scale = sum(work(i) for i in range(len(cases))) / sum(work(i) for i in idx)
    return t * scale, f"oracle on {k} of {len(cases)} matrices (setup + 1 and + 2 updates each), scaled by n^3 x iterations"


def run_batched(args):
    import torch

    from paper_1703_02283_gb300 import pthroot as P
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        cases, ps = batched_cases(args.count)
        its = [predicted_iterations(c, p, args.tol) for c, p in zip(cases, ps)]
        vals = []
        for _ in range(args.warmup + args.steps):
            v, what = oracle_batched_sample(cases, ps, its)
            vals.append(v)
        value = float(np.mean(vals[args.warmup:]))
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": value,
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": batched_config(args),
                          "cpu_baseline": {"value": value, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                                           "sample": what},
                          "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    import torch.distributed as dist
    world, rank, local = replica_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    cases, ps = batched_cases(args.count, rank)
    mats = [torch.from_numpy(c.A).to(dev) for c in cases]
    nbytes = sum(c.n * c.n * 8 for c in cases)

    # The batch (device memory, packed layout, captured solve graph) is created once; a step loads the 512
    # matrices into it, solves them all and copies every result out.
    b = P.pr_batch_init(mats, ps, P.pr_default_options(), stream.cuda_stream)
    P.pr_batch_set_timing(b, True)
    outs_dev = [torch.empty((c.n, c.n), dtype=torch.float64, device=dev) for c in cases]
    outs_host = [torch.empty((c.n, c.n), dtype=torch.float64).pin_memory() for c in cases]

    def one(inputs):
        s0 = P.pr_batch_stats(b)
        P.pr_batch_load(b, inputs)
        its, sts = P.pr_batch_solve(b, len(cases), P.PR_EMU64, args.tol)
        outs = outs_dev if inputs is mats else outs_host
        for i, C in enumerate(outs):
            P.pr_batch_result(b, i, C)
        s1 = P.pr_batch_stats(b)
        bst = {k: (s1[k] - s0[k] if k != "emu_slices" else s1[k]) for k in s1}
        return its, sts, outs, bst

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        one(mats)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        runs = [one(mats) for _ in range(args.steps)]
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, dev)
    its, sts, outs, bst = runs[-1]
    launches = sum(r[3]["launches"] for r in runs)
    # Roofline of the product kernel over the timed steps (CUDA events around every product launch).
    stage_ms = sum(r[3]["stage_ms"] for r in runs)
    stage_fl = sum(r[3]["stage_flops_timed"] for r in runs)
    stages = sum(r[3]["stages_timed"] for r in runs)
    S = bst["emu_slices"]
    pairs = S * (S + 1) // 2
    peaks, peak_src = load_peaks()
    roofline = {"bound": "tensor", "kernel": "k_gemm_emu (tcgen05 FP16 digit-slice products, batched work lists)",
                "achieved": stage_fl * pairs / (stage_ms * 1e-3) / 1e12, "peak": peaks["bf16_tflops_sustained"],
                "unit": "TFLOP/s", "traffic": None,
                "note": f"algorithmic = the {pairs} FP16 digit-pair products per emulated FP64 product (S={S}) of "
                        "every matrix's upper-triangle (or full) product; ragged tiles padded to 128 are not counted",
                "fp64_equivalent_tflops": stage_fl / (stage_ms * 1e-3) / 1e12,
                "peak_source": f"{peak_src} bf16 sustained x nominal fp16/bf16 ratio 1 (kernel timed inside a long step)",
                "launches_timed": stages, "avg_launch_ms": stage_ms / stages if stages else None,
                "product_kernel_share": stage_ms / (ms * args.steps)}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    errs = []
    for i, c in enumerate(cases):
        Z = (c.Q * c.lam ** (-1.0 / ps[i])) @ c.Q.T
        errs.append(float(np.linalg.norm(outs[i].cpu().numpy() - Z) / np.linalg.norm(Z)))
    e2e = None
    if not args.no_e2e:
        host = [c.A.copy() for c in cases]
        host = [torch.from_numpy(h).pin_memory() for h in host]
        barrier()
        t0 = time.perf_counter()
        one(host)
        barrier()
        e2e = {"value": max_over_ranks((time.perf_counter() - t0) * 1e3, dist, dev), "unit": "ms",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    P.pr_batch_destroy(b)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, what = oracle_batched_sample(cases, ps, its)
        cpu = {"value": v, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle", "sample": what}
    stat = {}
    for s_ in sts:
        stat[P.STATUS_NAMES[s_]] = stat.get(P.STATUS_NAMES[s_], 0) + 1
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "emu64(fp16 slices)", "data": "synthetic", "config": batched_config(args),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "batch": {"statuses": stat, "iterations_max": max(its), "iterations_mean": float(np.mean(its)),
                      "rel_error_median": float(np.median(errs)), "rel_error_max": float(np.max(errs)),
                      "matrices_per_second": world * len(cases) / (ms * 1e-3)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- learned initial guess

def learned_config(args):
    n = args.learned_n
    return {"workload": f"learned initial guess: overlap-like SPD S_ij = exp(-|r_i - r_j|/l), n={n} points uniform in a "
                        f"box of side {20 * (n / 2048) ** (1 / 3):.3g} l, jitter N(0, (0.01 l)^2) per coordinate and step, "
                        f"200 steps per sequence; MLP 8-64-64-4 (FP32) trained on {args.train_seqs} sequences sampled "
                        f"every {args.every} steps; timed on {args.test_seqs} held-out sequences sampled the same way; "
                        f"p=2, tol {args.tol:g}, gated polynomial C_0 (fallback Eq.3), PR_EMU64 products",
            "n": n, "p": 2, "train_sequences": args.train_seqs, "test_sequences": args.test_seqs, "every": args.every,
            "mode": "emu64", "l2": l2_note(handle_bytes(n)) + " per handle"}


def learned_sets(args):
    from paper_1703_02283_gb300 import learned as L
    n = args.learned_n
    train = [S for q in range(args.train_seqs) for S in L.overlap_sequence(q, 200, n, every=args.every)]
    test = [S for q in range(40, 40 + args.test_seqs) for S in L.overlap_sequence(q, 200, n, every=args.every)]
    return train, test


def run_learned(args):
    p = 2
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        from oracle import pthroot_oracle as O
        _, test = learned_sets(args)
        vals, what = [], ""
        for _ in range(args.warmup + args.steps):
            # The plain method on every test matrix: oracle setup + 1, 2 updates on one, extrapolated to the
            # iterations the scalar recurrence of Eq. 1 predicts for each matrix's spectrum.
            S0 = test[0]
            t0 = time.perf_counter()
            O.solve(S0, p, tol=0.0, max_iter=1, stag_below=0.0)
            t1 = time.perf_counter()
            O.solve(S0, p, tol=0.0, max_iter=2, stag_below=0.0)
            t2 = time.perf_counter()
            per = max((t2 - t1) - (t1 - t0), 1e-9)
            setup = max((t1 - t0) - per, 0.0)
            tot = 0.0
            for S in test:
                lam = np.linalg.eigvalsh(S)
                r = O.scalar_residuals(lam, lam / (O.norm_1(S) * O.norm_inf(S)), p, 200)
                hit = np.nonzero(r <= max(args.tol, 1e-13))[0]
                tot += setup + per * (int(hit[0]) if len(hit) else 200)
            vals.append(tot * 1e3)
            what = (f"oracle (plain method, Eq.3 C_0) setup + 1 and + 2 updates on one n={args.learned_n} matrix, "
                    f"extrapolated to the predicted iterations of each of the {len(test)} test matrices")
        value = float(np.mean(vals[args.warmup:]))
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": value,
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": learned_config(args),
                          "cpu_baseline": {"value": value, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                                           "sample": what},
                          "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch

    from paper_1703_02283_gb300 import learned as L
    from paper_1703_02283_gb300 import pthroot as P
    import torch.distributed as dist
    world, rank, local = replica_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream
    n = args.learned_n
    train, test = learned_sets(args)
    # Training (outside the timed region): labels from the plain method's converged roots, Adam on the device.
    t0 = time.perf_counter()
    samples = L.make_samples(torch, train, p, sptr, tol=args.tol)
    model = L.train(samples, steps=600, lr=3e-3, stream=sptr)
    train_s = time.perf_counter() - t0
    mlp = P.pr_mlp_create(model.params, 1, sptr)
    Ad = [torch.from_numpy(S).to(dev) for S in test]
    Cd = [torch.empty((n, n), dtype=torch.float64, device=dev) for _ in test]
    h = P.pr_init(Ad[0], n, p, P.pr_default_options(), sptr)
    P.pr_set_timing(h, True)

    def learned_step(inputs, outs):
        info = []
        for Ai, Co in zip(inputs, outs):
            P.pr_load(h, Ai)
            info.append(L.solve_learned(h, mlp, P.PR_EMU64, args.tol))
            P.pr_result(h, Co)
        return info

    def plain_step(inputs, outs):
        info = []
        for Ai, Co in zip(inputs, outs):
            P.pr_load(h, Ai)
            st, its = P.pr_iterate(h, 100, P.PR_EMU64, args.tol)
            P.pr_result(h, Co)
            info.append((st, its, P.PR_C0_EQ3, 0.0))
        return info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        learned_step(Ad, Cd)
    barrier()
    s0 = P.pr_stats(h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            info = learned_step(Ad, Cd)
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, dev)
    s1 = P.pr_stats(h)
    launches = (s1["launches"] - s0["launches"]) + args.steps * len(test)  # + one MLP forward per matrix
    dms = s1["gemm_ms_by_precision"][P.PR_EMU64] - s0["gemm_ms_by_precision"][P.PR_EMU64]
    dfl = s1["gemm_flops_by_precision"][P.PR_EMU64] - s0["gemm_flops_by_precision"][P.PR_EMU64]
    dn = s1["gemms_timed_by_precision"][P.PR_EMU64] - s0["gemms_timed_by_precision"][P.PR_EMU64]
    S = s1["emu_slices"]
    pairs = S * (S + 1) // 2
    peaks, peak_src = load_peaks()
    roofline = {"bound": "tensor", "kernel": "k_gemm_emu (tcgen05 FP16 digit-slice products)",
                "achieved": dfl * pairs / (dms * 1e-3) / 1e12, "peak": peaks["bf16_tflops_sustained"],
                "unit": "TFLOP/s", "traffic": None,
                "note": f"algorithmic = the {pairs} FP16 digit-pair products per emulated FP64 product (S={S})",
                "fp64_equivalent_tflops": dfl / (dms * 1e-3) / 1e12,
                "peak_source": f"{peak_src} bf16 sustained x nominal fp16/bf16 ratio 1 (kernel timed inside a long step)",
                "launches_timed": dn, "avg_launch_ms": dms / dn if dn else None,
                "product_kernel_share": dms / (ms * args.steps)}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    learned_out = [C.cpu().numpy() for C in Cd]

    # The plain method (Eq. 3 C_0) on the same matrices: the comparison.
    plain_step(Ad, Cd)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    pinfo = plain_step(Ad, Cd)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    pms = ev0.elapsed_time(ev1)
    plain_out = [C.cpu().numpy() for C in Cd]

    # Forward errors against an eigendecomposition root on the first two test matrices.
    errs_l, errs_p = [], []
    for i in range(min(2, len(test))):
        lam, V = np.linalg.eigh(test[i])
        Z = (V * lam ** (-1.0 / p)) @ V.T
        errs_l.append(float(np.linalg.norm(learned_out[i] - Z) / np.linalg.norm(Z)))
        errs_p.append(float(np.linalg.norm(plain_out[i] - Z) / np.linalg.norm(Z)))

    e2e = None
    if not args.no_e2e:
        Ah = [torch.from_numpy(S).pin_memory() for S in test]
        Ch = [torch.empty((n, n), dtype=torch.float64).pin_memory() for _ in test]
        learned_step(Ah, Ch)
        barrier()
        t0 = time.perf_counter()
        learned_step(Ah, Ch)
        barrier()
        nbytes = n * n * 8 * len(test)
        e2e = {"value": max_over_ranks((time.perf_counter() - t0) * 1e3, dist, dev), "unit": "ms",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        its_plain = [x[1] for x in pinfo]
        est, what = oracle_sample(test[0], p, int(np.mean(its_plain)))
        cpu = {"value": est * len(test), "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": what + f", times {len(test)} matrices (plain method, Eq.3 C_0)"}
    P.pr_destroy(h)
    P.pr_mlp_destroy(mlp)
    its_l = [x[1] for x in info]
    its_p = [x[1] for x in pinfo]
    used = sum(1 for x in info if x[2] == P.PR_C0_POLY)
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "emu64(fp16 slices)", "data": "synthetic", "config": learned_config(args),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "learned": {"matrices": len(test), "guess_used": used, "gate_values": [round(x[3], 4) for x in info],
                        "iterations_mean": float(np.mean(its_l)), "iterations": its_l,
                        "statuses": [P.STATUS_NAMES[x[0]] for x in info],
                        "rel_error_vs_eigh": errs_l, "training_samples": len(samples),
                        "training_loss_first_last": [model.loss_history[0], model.loss_history[-1]],
                        "training_seconds": train_s},
            "plain_eq3": {"ms_per_step": pms, "speedup_of_value": pms / ms, "iterations_mean": float(np.mean(its_p)),
                          "iterations": its_p, "statuses": [P.STATUS_NAMES[x[0]] for x in pinfo],
                          "rel_error_vs_eigh": errs_p}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    ps = [int(x) for x in args.p.split(",")]
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.impl == "reference":
        return run_reference(args, ps)

    import torch
    import torch.distributed as dist

    from paper_1703_02283_gb300 import pthroot as P

    world, rank, local = replica_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream

    # Replicas: every rank solves its own matrix of the same recipe (seed offset by rank).
    case = W.spd_from_spectrum(args.n, args.lam_min, replica_seed(args.seed, rank))
    A = torch.from_numpy(case.A).to(dev)
    C = torch.empty_like(A)
    opts = P.pr_default_options()
    opts.emu_slices = args.emu_slices
    handles = {p: P.pr_init(A, args.n, p, opts, sptr) for p in ps}

    def plan(p, mode):
        """(bulk precision, bulk steps, final precision) of one solve."""
        if mode == "fp64":
            return P.PR_FP64, 0, P.PR_FP64
        if mode == "emu64" or p != 1:
            return P.PR_EMU64, 0, P.PR_EMU64
        return P.PR_BF16, 100, P.PR_EMU64

    def solve_all(mode, Ain, Cout):
        info = {}
        for p, h in handles.items():
            bulk, nb, fin = plan(p, mode)
            P.pr_load(h, Ain)
            st, steps = P.pr_solve(h, bulk, nb, fin, args.tol)
            res = P.pr_residual(h, fin)
            P.pr_result(h, Cout)
            s = P.pr_stats(h)
            info[p] = {"status": P.STATUS_NAMES[st], "iterations": steps, "true_residual": res,
                       "iterations_by_precision": {PREC_NAMES[k]: s["iterations_by_precision"][k] for k in (0, 1, 3)
                                                   if s["iterations_by_precision"][k]},
                       "switch_iteration": s["switch_iteration"]}
        return info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def rel_err(Ct, p):
        Z = (case.Q * case.lam ** (-1.0 / p)) @ case.Q.T
        return float(np.linalg.norm(Ct.cpu().numpy() - Z) / np.linalg.norm(Z))

    for _ in range(args.warmup):
        solve_all(args.mode, A, C)
    barrier()
    s0 = {p: P.pr_stats(h) for p, h in handles.items()}
    for h in handles.values():
        P.pr_set_timing(h, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        infos = [solve_all(args.mode, A, C) for _ in range(args.steps)]
        ev1.record(stream)
        barrier()
    for h in handles.values():
        P.pr_set_timing(h, False)
    ms = ev0.elapsed_time(ev1) / args.steps
    s1 = {p: P.pr_stats(h) for p, h in handles.items()}
    ms = max_over_ranks(ms, dist, dev)
    last = infos[-1]
    for p, h in handles.items():
        P.pr_result(h, C)
        last[p]["rel_error_vs_closed_form"] = rel_err(C, p)
    launches = sum(s1[p]["launches"] - s0[p]["launches"] for p in ps)

    # Roofline of the dominant product kernel over the timed region (CUDA events around every launch).
    def delta(key, k):
        return sum(s1[p][key][k] - s0[p][key][k] for p in ps)

    by_prec = {k: (delta("gemm_ms_by_precision", k), delta("gemm_flops_by_precision", k),
                   delta("gemms_timed_by_precision", k)) for k in (0, 1, 3)}
    dom = max(by_prec, key=lambda k: by_prec[k][0])
    dms, dfl, dn = by_prec[dom]
    peaks, peak_src = load_peaks()
    S = s1[ps[0]]["emu_slices"]
    if dom == P.PR_EMU64:
        pairs = S * (S + 1) // 2
        exec_fl = dfl * pairs
        # DRAM bytes (read + write) per symmetric n = 4096 product from one ncu capture; other sizes were not
        # captured.
        traffic_seen = EMU_TRAFFIC_BYTES.get(args.n) if S == 8 else None
        roofline = {"bound": "tensor", "kernel": "k_gemm_emu (tcgen05 FP16 digit-slice products)",
                    "achieved": exec_fl / (dms * 1e-3) / 1e12, "peak": peaks["bf16_tflops_sustained"],
                    "unit": "TFLOP/s", "traffic": None, "traffic_last_capture": traffic_seen,
                    "note": f"algorithmic = the {pairs} FP16 digit-pair products per emulated FP64 product "
                            f"(S={S}), upper-triangle tiles; fp64_equivalent_tflops = FP64 flops / time",
                    "fp64_equivalent_tflops": dfl / (dms * 1e-3) / 1e12,
                    "peak_source": f"{peak_src} bf16 sustained x nominal fp16/bf16 ratio 1 (kernel timed inside a long step)"}
    elif dom == P.PR_BF16:
        roofline = {"bound": "tensor", "kernel": "k_gemm_bf16_tc", "achieved": dfl / (dms * 1e-3) / 1e12,
                    "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s", "traffic": None,
                    "peak_source": f"{peak_src} bf16 sustained"}
    else:
        peak = peaks["bf16_tflops_sustained"] * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
        roofline = {"bound": "tensor", "kernel": "k_gemm_f64 (DMMA)", "achieved": dfl / (dms * 1e-3) / 1e12,
                    "peak": peak, "unit": "TFLOP/s", "traffic": None,
                    "peak_source": f"{peak_src} bf16 sustained x nominal fp64/bf16 ({NOMINAL_FP64_TFLOPS}/"
                                   f"{NOMINAL_BF16_TFLOPS})"}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    roofline.update({"launches_timed": dn, "avg_launch_ms": dms / dn if dn else None,
                     "flops_per_launch_fp64_equivalent": dfl / dn if dn else None})
    kernel_share = {PREC_NAMES[k]: round(v[0] / (ms * args.steps), 4) for k, v in by_prec.items() if v[2]}

    # End to end through pinned host buffers, copies inside the timed region.
    e2e = None
    if not args.no_e2e:
        Ah = torch.from_numpy(case.A).pin_memory()
        Ch = torch.empty_like(Ah).pin_memory()
        solve_all(args.mode, Ah, Ch)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            solve_all(args.mode, Ah, Ch)
        barrier()
        nbytes = args.n * args.n * 8 * len(ps)
        e2e = {"value": max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, dist, dev), "unit": "ms",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # The plain FP64 GPU iteration on the same matrices, once per p (the speed comparison).
    plain = None
    if not args.no_compare and args.mode != "fp64":
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        pinfo = solve_all("fp64", A, C)
        e1.record(stream)
        barrier()
        for p, h in handles.items():
            P.pr_result(h, C)
            pinfo[p]["rel_error_vs_closed_form"] = rel_err(C, p)
        pms = e0.elapsed_time(e1)
        plain = {"ms_per_step": pms, "speedup_of_value": pms / ms, "solves": {str(p): v for p, v in pinfo.items()}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tot, what = 0.0, []
        for p in ps:
            est, w = oracle_sample(case.A, p, last[p]["iterations"])
            tot += est
            what.append(w)
        cpu = {"value": tot, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle", "sample": "; ".join(what)}

    for h in handles.values():
        P.pr_destroy(h)
    if rank == 0:
        line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fast": "bf16+emu64(fp16 slices)", "emu64": "emu64(fp16 slices)",
                                               "fp64": "f64"}[args.mode],
                "data": "synthetic", "config": config_dict(args, ps), "roofline": roofline,
                "kernel_time_share": kernel_share, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "solves": {str(p): v for p, v in last.items()}, "plain_fp64_gpu": plain}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
