"""Benchmark: time to an FP64-accurate A^{-1/p} on one GB300, through the library's C ABI.

Workload: the n = 4096, kappa = 1e3 SPD matrix (Q diag(lam) Q^T, lam log-uniform in [1e-3, 1], seed 1),
roots p = 1, 2, 3, 4, initial guess of Eq. 3, tolerance 1e-12 on the iteration's residual.

One step = the whole hot path for every p in --p: load A (checks, ||A||_1, ||A||_inf, C_0), iterate Eq. 1
to the tolerance or the precision floor (the coupled form's stop verified against the true residual), the
true residual ||I - C^p A||_F and the result copy. The value is milliseconds per step (lower is better) for
--mode:
  fast   FP64-accurate products from exact FP16 digit slices (PR_EMU64) for every p; for p = 1, whose
         Newton-Schulz form corrects earlier errors, BF16 iterations first, then PR_EMU64 ones; for p >= 2,
         whose coupled form keeps the error of its iterates, Newton refinement afterwards (pr_refine: EMU64
         residuals, BF16 conjugate-gradient solves) (default);
  emu64  PR_EMU64 for every iteration;
  fp64   native FP64 products (the plain FP64 GPU iteration).
Beside the value the line reports the same solves from the scaled identity C_0 = ||A||_1^{-1/p} I (Sec. 2's
"other choices" of C_0; FP64-accurate for every p, where Eq. 3's C_0 loses u kappa^(p+1)), timed the same
way, and, unless --no-compare, the plain FP64 GPU iteration of both (--compare-warmup + --compare-steps
steps each). Unless --no-extra it also runs the batched workload (512 matrices) and the learned-guess
workload with --sub-warmup / --sub-steps steps and reports them under "batched" and "learned". Inputs are
resident in HBM before the timed regions; the working sets exceed the 129 MB L2.

`--impl reference` times the CPU oracle (numpy FP64) on the host cores instead: each step times one oracle
update of one root (the roots in turn); the value is the oracle's time to the same solves, the measured
setup plus the measured update time times the iteration count, and one full p = 1 oracle solve checks that
model. ms_per_step is the measured time of a step.
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
PREC_NAMES = {0: "fp64", 1: "emu64", 2: "fp32x", 3: "bf16", 4: "fp8"}
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one symmetric product of the kernel as it is now, by n
# (profiles/k_gemm_emu_n4096.md). A change to the kernel empties this until it is captured again.
EMU_TRAFFIC_CURRENT: dict = {4096: 2.687357e9 + 0.348960e9}
# Mode fast, p >= 2: Newton refinement after the EMU64 iterations (pr_refine: EMU64 residuals, BF16 conjugate-
# gradient solves, each correction about a hundredfold).
REFINE = dict(max_steps=12, cg_max=40, cg_tol=1e-2)


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
    ap.add_argument("--workload", default="single", choices=["single", "batched", "learned", "f1", "f3"],
                    help="single: the n=4096 matrix for every p; batched: 512 matrices, n in [64, 1024]")
    ap.add_argument("--count", type=int, default=512, help="batched: number of matrices")
    ap.add_argument("--learned-n", type=int, default=2048, help="learned: matrix order")
    ap.add_argument("--train-seqs", type=int, default=40, help="learned: training sequences (ids 0..)")
    ap.add_argument("--test-seqs", type=int, default=10, help="learned: held-out sequences (ids 40..)")
    ap.add_argument("--every", type=int, default=10, help="learned: sample every this many of 200 steps")
    ap.add_argument("--compare-steps", type=int, default=2, help="timed steps of each plain FP64 comparison")
    ap.add_argument("--compare-warmup", type=int, default=1, help="warm-up steps of each plain FP64 comparison")
    ap.add_argument("--no-scaled-identity", action="store_true", help="skip the scaled-identity arm")
    ap.add_argument("--no-refine", action="store_true",
                    help="mode fast: skip the Newton refinement (pr_refine) of the p >= 2 solves")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and learned summaries")
    ap.add_argument("--sub-steps", type=int, default=5, help="timed steps of the batched / learned summaries")
    ap.add_argument("--sub-warmup", type=int, default=3, help="warm-up steps of the batched / learned summaries")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end measurement")
    ap.add_argument("--f1-n", type=int, default=768, help="f1: order of the overlap stand-in")
    ap.add_argument("--f1-iters", type=int, default=40, help="f1: iterations per mantissa width")
    ap.add_argument("--f1-storage-bits", default="2,3,4,6,8,10,12,16,20,24")
    ap.add_argument("--f1-arith-bits", default="6,8,9,10,11,12,14,16,18,20,24")
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

class OracleModel:
    """Time of the oracle's solve of (A, p) from measurements: its setup (norms, C_0 and, for the coupled
    form, M_0 = C_0^p A) once, and the time of single updates, measured on the oracle's own iterates."""

    def __init__(self, A: np.ndarray, p: int, c0: str = "eq3"):
        from oracle import pthroot_oracle as O
        self.O, self.A, self.p, self.c0 = O, A, p, c0
        self.form = O.default_form(p)
        t0 = time.perf_counter()
        C = O.initial_guess_eq3(A) if c0 == "eq3" else O.initial_guess_scaled_identity(A, p)
        if self.form == "coupled":
            self.X, self.M = O.coupled_start(C, A, p)
            np.linalg.norm(np.eye(A.shape[0]) - self.M)
        else:
            self.C = C
        self.setup_s = time.perf_counter() - t0
        self.updates = []

    def time_update(self) -> float:
        """One update of the oracle's form, with the residual it tests (seconds)."""
        O, A, n = self.O, self.A, self.A.shape[0]
        t0 = time.perf_counter()
        if self.form == "coupled":
            self.X, self.M = O.step_coupled(self.X, self.M, self.p)
            np.linalg.norm(np.eye(n) - self.M)
        else:
            T = A @ self.C
            np.linalg.norm(np.eye(n) - T)
            self.C = O.symmetrize(2.0 * self.C - self.C @ T)
        dt = time.perf_counter() - t0
        self.updates.append(dt)
        return dt

    def solve_ms(self, iterations: int) -> float:
        return (self.setup_s + float(np.median(self.updates)) * iterations) * 1e3


def oracle_sample(A: np.ndarray, p: int, iterations: int) -> tuple[float, str]:
    """The oracle's time to a solve of `iterations` updates: measured setup + iterations x a measured update."""
    m = OracleModel(A, p)
    m.time_update()
    return m.solve_ms(iterations), (f"n={A.shape[0]} p={p}: oracle setup + one update measured, times "
                                    f"{iterations} updates")


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
            "refine": None if args.mode != "fast" or args.no_refine else
            {"p": ">= 2", "residual": "emu64", "solve": "bf16", **REFINE},
            "l2": l2_note(handle_bytes(args.n)) + " per handle"}


def run_reference(args, ps):
    """The oracle timed on the host cores. Each step times one update of one root (the roots in turn, on the
    oracle's own iterates); the value is the modelled time of the oracle's solves of every root (measured
    setup + median measured update x the iterations the exact-arithmetic recurrence predicts). Before the
    steps, one full p = 1 oracle solve is timed and compared with the model (model_check)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from oracle import pthroot_oracle as O
    case = W.spd_from_spectrum(args.n, args.lam_min, args.seed)
    its = {p: predicted_iterations(case, p, args.tol) for p in ps}
    check = None
    if 1 in ps:
        _, info = O.solve(case.A, 1, tol=args.tol)
        m1 = OracleModel(case.A, 1)
        for _ in range(2):
            m1.time_update()
        check = {"p": 1, "full_solve_ms": info.seconds * 1e3, "iterations": info.iterations,
                 "model_ms": m1.solve_ms(info.iterations)}
        check["model_over_full"] = check["model_ms"] / check["full_solve_ms"]
    models = {p: OracleModel(case.A, p) for p in ps}
    step_ms = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        models[ps[k % len(ps)]].time_update()
        step_ms.append((time.perf_counter() - t0) * 1e3)
    for p in ps:  # a root whose update fell only into the warm-up steps still gets a measured update
        if not models[p].updates:
            models[p].time_update()
    value = sum(models[p].solve_ms(its[p]) for p in ps)
    ms = float(np.mean(step_ms[args.warmup:])) if args.steps else 0.0
    sample = (f"n={args.n}, p={','.join(map(str, ps))}: oracle setup of every root and single updates measured "
              f"(one per step, roots in turn), value = setup + median update x predicted iterations "
              f"({', '.join(f'p={p}: {its[p]}' for p in ps)}); the iteration of Eq. 1 only: the GPU arm's "
              f"refinement of the p >= 2 roots (Newton steps with conjugate-gradient solves) has no oracle time here")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, ps),
            "value_model": "value = modelled oracle time to the solves of one step; ms_per_step = measured time of "
                           "one benchmark step (one oracle update)",
            "model_check": check,
            "cpu_baseline": {"value": value, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
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
        vals, step_ms = [], []
        for _ in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            v, what = oracle_batched_sample(cases, ps, its)
            step_ms.append((time.perf_counter() - t0) * 1e3)
            vals.append(v)
        value = float(np.mean(vals[args.warmup:]))
        ms = float(np.mean(step_ms[args.warmup:])) if args.steps else 0.0
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "value_model": "value = modelled oracle time to every solve of the batch; ms_per_step = "
                                         "measured time of one benchmark step (the sampled oracle updates)",
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
    line = measure_batched(args, world, rank, local, dist, args.steps, args.warmup, not args.no_e2e,
                           rank == 0 and world == 1 and not args.no_cpu_baseline)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_batched(args, world, rank, local, dist, steps, warmup, e2e_on, cpu_on):
    """The batched workload's JSON fields on this rank (timed over `steps` steps after `warmup`)."""
    import torch

    from paper_1703_02283_gb300 import pthroot as P
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

    for _ in range(warmup):
        one(mats)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        runs = [one(mats) for _ in range(steps)]
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, dist, dev)
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
                "product_kernel_share": stage_ms / (ms * steps)}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    errs = []
    for i, c in enumerate(cases):
        Z = (c.Q * c.lam ** (-1.0 / ps[i])) @ c.Q.T
        errs.append(float(np.linalg.norm(outs[i].cpu().numpy() - Z) / np.linalg.norm(Z)))
    tres = [P.pr_batch_matrix(b, i)["true_residual"] for i in range(len(cases))]


    e2e = None
    if e2e_on:
        host = [c.A.copy() for c in cases]
        host = [torch.from_numpy(h).pin_memory() for h in host]
        barrier()
        t0 = time.perf_counter()
        one(host)
        barrier()
        e2e = {"value": max_over_ranks((time.perf_counter() - t0) * 1e3, dist, dev), "unit": "ms",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    P.pr_batch_destroy(b)

    # The same batch from the scaled identity C_0 = ||A||_1^{-1/p} I (reading of Sec. 2's "other choices"): its
    # M_0 spans kappa instead of kappa^(p+1), so every matrix ends FP64 accurate, in fewer iterations.
    o_si = P.pr_default_options()
    o_si.c0 = P.PR_C0_SCALED_I
    b_si = P.pr_batch_init(mats, ps, o_si, stream.cuda_stream)
    try:
        def one_si():
            P.pr_batch_load(b_si, mats)
            r = P.pr_batch_solve(b_si, len(cases), P.PR_EMU64, args.tol)
            for i, C in enumerate(outs_dev):
                P.pr_batch_result(b_si, i, C)
            return r
        one_si()
        barrier()
        es0, es1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es0.record(stream)
        for _ in range(steps):
            its_si, sts_si = one_si()
        es1.record(stream)
        barrier()
        errs_si = []
        for i, c in enumerate(cases):
            Z = (c.Q * c.lam ** (-1.0 / ps[i])) @ c.Q.T
            errs_si.append(float(np.linalg.norm(outs_dev[i].cpu().numpy() - Z) / np.linalg.norm(Z)))
        si = {"value": max_over_ranks(es0.elapsed_time(es1) / steps, dist, dev), "unit": "ms", "steps": steps,
              "statuses": {P.STATUS_NAMES[k]: int(v) for k, v in zip(*np.unique(sts_si, return_counts=True))},
              "iterations_mean": float(np.mean(its_si)), "rel_error_median": float(np.median(errs_si)),
              "rel_error_max": float(np.max(errs_si))}
    finally:
        P.pr_batch_destroy(b_si)
    cpu = None
    if cpu_on:
        v, what = oracle_batched_sample(cases, ps, its)
        cpu = {"value": v, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle", "sample": what}
    stat = {}
    for s_ in sts:
        stat[P.STATUS_NAMES[s_]] = stat.get(P.STATUS_NAMES[s_], 0) + 1
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "emu64(fp16 slices)", "data": "synthetic", "config": batched_config(args),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "batch": {"statuses": stat, "iterations_max": max(its), "iterations_mean": float(np.mean(its)),
                      "rel_error_median": float(np.median(errs)), "rel_error_max": float(np.max(errs)),
                      "true_residual_median": float(np.median(tres)), "true_residual_max": float(np.max(tres)),
                      "matrices_per_second": world * len(cases) / (ms * 1e-3)},
            "scaled_identity": si}
    return line


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
    """(training matrices as a generator, one sequence at a time; held-out test matrices as a list)."""
    from paper_1703_02283_gb300 import learned as L
    n = args.learned_n
    train = (S for q in range(args.train_seqs) for S in L.overlap_sequence(q, 200, n, every=args.every))
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
        # The plain method on every test matrix: the iterations the scalar recurrence of Eq. 1 predicts for
        # each matrix's spectrum, at the oracle's measured setup and update times on the first one.
        predicted = []
        for S in test:
            lam = np.linalg.eigvalsh(S)
            r = O.scalar_residuals(lam, lam / (O.norm_1(S) * O.norm_inf(S)), p, 200)
            hit = np.nonzero(r <= max(args.tol, 1e-13))[0]
            predicted.append(int(hit[0]) if len(hit) else 200)
        model = OracleModel(test[0], p)
        step_ms = []
        for _ in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            model.time_update()
            step_ms.append((time.perf_counter() - t0) * 1e3)
        value = sum(model.solve_ms(k) for k in predicted)
        ms = float(np.mean(step_ms[args.warmup:])) if args.steps else 0.0
        what = (f"oracle (plain method, Eq.3 C_0): setup and one update per step measured on one n={args.learned_n} "
                f"matrix, times the predicted iterations of each of the {len(test)} test matrices")
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "value_model": "value = modelled oracle time to every test solve; ms_per_step = measured "
                                         "time of one benchmark step (one oracle update)",
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": learned_config(args),
                          "cpu_baseline": {"value": value, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                                           "sample": what},
                          "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    import torch.distributed as dist
    world, rank, local = replica_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    line = measure_learned(args, world, rank, local, dist, args.steps, args.warmup, not args.no_e2e,
                           rank == 0 and world == 1 and not args.no_cpu_baseline)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_learned(args, world, rank, local, dist, steps, warmup, e2e_on, cpu_on):
    """The learned-guess workload's JSON fields on this rank (timed over `steps` steps after `warmup`)."""
    import torch

    from paper_1703_02283_gb300 import learned as L
    from paper_1703_02283_gb300 import pthroot as P
    p = 2
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

    for _ in range(warmup):
        learned_step(Ad, Cd)
    barrier()
    s0 = P.pr_stats(h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            info = learned_step(Ad, Cd)
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, dist, dev)
    s1 = P.pr_stats(h)
    launches = (s1["launches"] - s0["launches"]) + steps * len(test)  # + one MLP forward per matrix
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
                "product_kernel_share": dms / (ms * steps)}
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
    if e2e_on:
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
    if cpu_on:
        its_plain = [x[1] for x in pinfo]
        est, what = oracle_sample(test[0], p, int(np.mean(its_plain)))
        cpu = {"value": est * len(test), "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": what + f", times {len(test)} matrices (plain method, Eq.3 C_0)"}
    P.pr_destroy(h)
    P.pr_mlp_destroy(mlp)
    its_l = [x[1] for x in info]
    its_p = [x[1] for x in pinfo]
    used = sum(1 for x in info if x[2] == P.PR_C0_POLY)
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
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
    return line


# ----------------------------------------------------------------------------- the paper's precision experiment

def f1_matrix(n: int):
    """The overlap stand-in of the experiment (Sec. 4.3: N = 768, p = 2): n points uniform in a cube of side 20
    (kappa about 20 at n = 768, the recipe the survey probed), seeded 7000 + n, and its exact inverse square
    root from a LAPACK eigendecomposition (host)."""
    S = W.overlap_matrix(W.overlap_points(n, 20.0, 7000 + n))
    lam, V = np.linalg.eigh(S)
    return S, (V * lam ** -0.5) @ V.T


def f1_config(args):
    return {"workload": f"custom-precision experiment: overlap stand-in n={args.f1_n}, p=2, literal Eq. 1 from Eq. 3, "
                        f"{args.f1_iters} iterations per mantissa width, storage widths {args.f1_storage_bits}, "
                        f"arithmetic widths {args.f1_arith_bits}", "n": args.f1_n, "p": 2,
            "l2": l2_note(9 * 8.0 * args.f1_n ** 2) + " per handle"}


def measure_f1(args, local):
    """Per mode and mantissa width: the error ||C_k - S^{-1/2}||_F (absolute, as Fig. 2 plots it) of every
    iterate; reported are its smallest value, the iteration where it occurs and the final error. A width
    'converges' when the smallest error is below 1e-2 of the starting error."""
    import torch

    from paper_1703_02283_gb300 import pthroot as P
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    S, Z = f1_matrix(args.f1_n)
    A = torch.from_numpy(S).to(dev)
    C = torch.empty_like(A)
    zn = float(np.linalg.norm(Z))
    table = {}
    t0 = time.perf_counter()
    for mode, name, bits in ((P.PR_QUANT_STORAGE, "storage", args.f1_storage_bits),
                             (P.PR_QUANT_ARITH, "arithmetic", args.f1_arith_bits)):
        rows = []
        for m in [int(x) for x in bits.split(",")]:
            o = P.pr_default_options()
            o.form = P.PR_FORM_LITERAL
            o.quant_bits = m
            o.quant_mode = mode
            o.stag_below = 0.0
            h = P.pr_init(A, args.f1_n, 2, o, stream.cuda_stream)
            errs = []
            Zd = torch.from_numpy(Z).to(dev)
            try:
                for k in range(args.f1_iters + 1):
                    if k:
                        try:
                            P.pr_iterate(h, 1, P.PR_FP64, 0.0)
                        except P.PthrootError as exc:  # the iterate overflowed: the width diverged
                            if exc.status != P.PR_EDIVERGED:
                                raise
                            errs += [float("inf")] * (args.f1_iters + 1 - k)
                            break
                    P.pr_result(h, C)
                    e = float(torch.linalg.norm(C - Zd).item())
                    errs.append(e if np.isfinite(e) else float("inf"))
            finally:
                P.pr_destroy(h)
            k_min = int(np.argmin(errs))
            rows.append({"bits": m, "min_error": errs[k_min], "min_rel_error": errs[k_min] / zn, "at_iteration": k_min,
                         "final_error": errs[-1] if np.isfinite(errs[-1]) else "inf",
                         "converges": bool(errs[k_min] < 1e-2 * errs[0]),
                         "errors": [float(f"{e:.3g}") if np.isfinite(e) else "inf" for e in errs]})
        table[name] = rows
    torch.cuda.synchronize(dev)
    return {"value": (time.perf_counter() - t0) * 1e3, "table": table, "reference_norm": zn}


def measure_large(args, local):
    """The large recipe (n = 16384, kappa = 1e4, p = 2, the matrix built on the device, scaled-identity start):
    the FP8 -> BF16 -> split-FP32 ladder, the same ladder ending in EMU64, the split-FP32 rung refined by Newton
    corrections (pr_refine), and the all-EMU64 solve, each timed once after a short untimed pass
    that tunes and allocates. Errors: relative Frobenius error on a sampled 64 x 64 block of the closed form
    Q diag(lam^-1/2) Q^T (rows I, columns I) and the true residual of the library's own evaluation."""
    import torch

    from oracle import pthroot_oracle as O
    from paper_1703_02283_gb300 import pthroot as P
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    n, p = W.LARGE_CASE["n"], W.LARGE_CASE["p"]
    case = W.spd_from_spectrum_device(n, W.LARGE_CASE["lam_min"], W.LARGE_CASE["seed"], dev)
    rng = np.random.default_rng(16384)
    I = np.sort(rng.choice(n, 64, replace=False))
    QI = case.Q[I].cpu().numpy()
    Zb = O.closed_form_block(QI, QI, case.lam, p)
    del case.Q
    torch.cuda.empty_cache()
    out = {"workload": f"SPD n={n}, kappa=1e4, p={p}, scaled-identity C_0, tol {args.tol:g}"}
    for name, rungs, refine in (("ladder_fp8_bf16_fp32x", [P.PR_FP8, P.PR_BF16, P.PR_FP32X], False),
                                ("ladder_fp8_bf16_fp32x_emu64", [P.PR_FP8, P.PR_BF16, P.PR_FP32X, P.PR_EMU64], False),
                                ("ladder_fp32x_refined", [P.PR_FP32X], True),
                                ("emu64", [P.PR_EMU64], False)):
        o = P.pr_default_options()
        o.c0 = P.PR_C0_SCALED_I
        h = P.pr_init(case.A, n, p, o, stream.cuda_stream)
        try:
            for prec in rungs:  # tune and allocate outside the timed solve
                P.pr_iterate(h, 1, prec, args.tol)
            if refine:
                P.pr_refine(h, P.PR_EMU64, P.PR_BF16, 1, 0.0, REFINE["cg_max"], REFINE["cg_tol"])
            P.pr_load(h, case.A)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, steps = P.pr_solve_ladder(h, rungs, None, args.tol)
            if refine:  # the split-FP32 rung's end, refined: Newton corrections (EMU64 residuals, BF16 solves)
                st, _ = P.pr_refine(h, P.PR_EMU64, P.PR_BF16, REFINE["max_steps"], args.tol, REFINE["cg_max"],
                                    REFINE["cg_tol"])
            e1.record(stream)
            e1.synchronize()
            s = P.pr_stats(h)
            C = torch.empty((n, n), dtype=torch.float64, device=dev)
            P.pr_result(h, C)
            Cb = C[I][:, I].cpu().numpy()
            del C
        finally:
            P.pr_destroy(h)
        out[name] = {"ms": e0.elapsed_time(e1), "status": P.STATUS_NAMES[st], "iterations": steps,
                     "iterations_by_precision": {PREC_NAMES[k]: s["iterations_by_precision"][k]
                                                 for k in range(P.PR_NPREC) if s["iterations_by_precision"][k]},
                     "true_residual": s["true_residual"], "rungs_discarded": s["ladder_restores"],
                     "rel_error_sampled_block": float(np.linalg.norm(Cb - Zb) / np.linalg.norm(Zb))}
        if refine:
            out[name]["refine"] = {"steps": len(s["refine_residuals"]) - 1, "residuals": s["refine_residuals"],
                                   "cg_iterations": s["refine_cg"]}
        torch.cuda.empty_cache()
    return out


def measure_f3(args, local):
    """The sparse overlap stand-in of Sec. 4.1 at the paper's densities (6.2 % non-zeros at N = 3072, 3.1 % at
    6144): S^-1 (p = 1: BF16 then EMU64 Newton-Schulz) and S^-1/2 (p = 2: EMU64 coupled form from Eq. 3, then the
    refinement), each with block-sparse products with S (pr_options.block_sparse) and dense ones, one timed solve
    after an untimed one on the same handle. The two give bit-identical results; forward errors against a LAPACK
    root at N = 3072."""
    import torch

    from oracle import pthroot_oracle as O
    from paper_1703_02283_gb300 import pthroot as P
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    out = {}
    for n in (3072, 6144):
        S, cut = W.sparse_overlap(n, W.PAPER_OVERLAP_DENSITY[n], n)
        Sd = torch.from_numpy(S).to(dev)
        rec = {"density": float(np.count_nonzero(S) / S.size), "cutoff": cut}
        for p in (1, 2):
            Z = O.eig_root(S, p) if n <= 3072 else None
            res = {}
            for bs in (1, 0):
                o = P.pr_default_options()
                o.block_sparse = bs
                h = P.pr_init(Sd, n, p, o, stream.cuda_stream)
                try:
                    def solve():
                        P.pr_load(h, Sd)
                        if p == 1:
                            st, its = P.pr_solve(h, P.PR_BF16, 100, P.PR_EMU64, args.tol)
                        else:
                            st, its = P.pr_iterate(h, 100, P.PR_EMU64, args.tol)
                            st, _ = P.pr_refine(h, P.PR_EMU64, P.PR_BF16, REFINE["max_steps"], args.tol,
                                                REFINE["cg_max"], REFINE["cg_tol"])
                        return st, its
                    solve()
                    torch.cuda.synchronize(dev)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    st, its = solve()
                    e1.record(stream)
                    e1.synchronize()
                    s = P.pr_stats(h)
                    C = torch.empty((n, n), dtype=torch.float64, device=dev)
                    P.pr_result(h, C)
                finally:
                    P.pr_destroy(h)
                r = {"ms": e0.elapsed_time(e1), "status": P.STATUS_NAMES[st], "iterations": its,
                     "true_residual": s["true_residual"], "sparse_keep": s["sparse_keep"],
                     "sparse_products": s["sparse_products"]}
                if Z is not None:
                    r["rel_error_vs_lapack"] = O.forward_error(C.cpu().numpy(), Z)
                res["block_sparse" if bs else "dense"] = (r, C)
            (rs, Cs), (rd, Cd) = res["block_sparse"], res["dense"]
            rs["bit_identical_to_dense"] = bool(torch.equal(Cs, Cd))
            rs["speedup_over_dense"] = rd["ms"] / rs["ms"]
            rec[f"p{p}"] = {"block_sparse": rs, "dense": rd}
            del Cs, Cd
        out[str(n)] = rec
        del Sd
        torch.cuda.empty_cache()
    return out


def run_f1(args):
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        from oracle import pthroot_oracle as O
        S, Z = f1_matrix(args.f1_n)
        step_ms = []
        for _ in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            O.quantized_iterates(S, 2, 10, "storage", 1)
            step_ms.append((time.perf_counter() - t0) * 1e3)
        per = float(np.median(step_ms))
        widths = len(args.f1_storage_bits.split(",")) + len(args.f1_arith_bits.split(","))
        value = per * args.f1_iters * widths
        ms = float(np.mean(step_ms[args.warmup:])) if args.steps else 0.0
        print(json.dumps({"impl": "reference", "metric": "time of the custom-precision sweep", "value": value,
                          "unit": "ms", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f64", "data": "synthetic", "config": f1_config(args),
                          "value_model": "value = one oracle storage-mode iteration (measured per step) x iterations x "
                                         "widths; the arithmetic mode's per-operation rounding is slower still",
                          "cpu_baseline": {"value": value, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                                           "sample": f"one storage-mode iteration at n={args.f1_n}, m=10"},
                          "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    import torch
    world, rank, local = replica_env()
    torch.cuda.set_device(local)
    r = measure_f1(args, local)
    if rank == 0:
        print(json.dumps({"metric": "time of the custom-precision sweep", "value": r["value"], "unit": "ms",
                          "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": r["value"],
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "custom-m-bit",
                          "data": "synthetic", "config": f1_config(args), "f1": r["table"]}), flush=True)


def main():
    args = parse()
    ps = [int(x) for x in args.p.split(",")]
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "f1":
        return run_f1(args)
    if args.workload == "f3":  # the sparse overlap summary on its own (one GPU, rank 0 prints)
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the sparse overlap summary has no oracle timing"}))
            return None
        import torch
        torch.cuda.set_device(replica_env()[2])
        out = measure_f3(args, replica_env()[2])
        if replica_env()[1] == 0:
            print(json.dumps({"workload": "f3", **out}), flush=True)
        return None
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

    def make_handles(c0):
        handles = {}
        for p in ps:
            opts = P.pr_default_options()
            opts.emu_slices = args.emu_slices
            opts.c0 = c0
            # A refined solve is verified at the end of the refinement; the coupled form's own verification of
            # the iterate it hands over would be evaluated for nothing.
            opts.verify = 0 if (args.mode == "fast" and p >= 2 and not args.no_refine) else 1
            handles[p] = P.pr_init(A, args.n, p, opts, sptr)
        return handles

    arms = {"eq3": make_handles(P.PR_C0_EQ3)}
    if not args.no_scaled_identity:
        arms["scaled_identity"] = make_handles(P.PR_C0_SCALED_I)

    def plan(p, mode):
        """(bulk precision, bulk steps, final precision) of one solve."""
        if mode == "fp64":
            return P.PR_FP64, 0, P.PR_FP64
        if mode == "emu64" or p != 1:
            return P.PR_EMU64, 0, P.PR_EMU64
        return P.PR_BF16, 100, P.PR_EMU64

    def solve_all(handles, mode, Ain, Cout):
        info = {}
        for p, h in handles.items():
            bulk, nb, fin = plan(p, mode)
            P.pr_load(h, Ain)
            st, steps = P.pr_solve(h, bulk, nb, fin, args.tol)
            refine = None
            if mode == "fast" and p >= 2 and not args.no_refine:
                # The coupled form keeps the error its iterates picked up (Eq. 3's M_0 spans kappa^(p+1));
                # Newton corrections with BF16 solves remove it.
                st, k = P.pr_refine(h, P.PR_EMU64, P.PR_BF16, REFINE["max_steps"], args.tol, REFINE["cg_max"],
                                    REFINE["cg_tol"])
                refine = k
            s = P.pr_stats(h)
            # The true residual ||I - C^p A||_F of the result: evaluated by the library at the stop (the verified
            # coupled stop, the tested Newton-Schulz residual, or the end of the refinement).
            res = s["true_residual"]
            P.pr_result(h, Cout)
            info[p] = {"status": P.STATUS_NAMES[st], "iterations": steps, "true_residual": res,
                       "tol_met": bool(res <= args.tol),
                       "iterations_by_precision": {PREC_NAMES[k]: s["iterations_by_precision"][k]
                                                   for k in range(P.PR_NPREC) if s["iterations_by_precision"][k]},
                       "switch_iteration": s["switch_iteration"],
                       "emu_variant": {"sym": {"tile_n": s["emu_tile_n"][0], "split": s["emu_tile_split"][0]},
                                       "full": {"tile_n": s["emu_tile_n"][1], "split": s["emu_tile_split"][1]}}}
            if refine is not None:
                info[p]["refine"] = {"steps": refine, "residuals": s["refine_residuals"],
                                     "cg_iterations": s["refine_cg"]}
        return info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def rel_err(Ct, p):
        Z = (case.Q * case.lam ** (-1.0 / p)) @ case.Q.T
        return float(np.linalg.norm(Ct.cpu().numpy() - Z) / np.linalg.norm(Z))

    def timed(handles, mode, steps, warmup, sample_clocks=False):
        """(ms per step, the last step's solve records with forward errors, stats before and after)."""
        for _ in range(warmup):
            solve_all(handles, mode, A, C)
        barrier()
        s0 = {p: P.pr_stats(h) for p, h in handles.items()}
        for h in handles.values():
            P.pr_set_timing(h, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.__enter__()
        try:
            barrier()
            ev0.record(stream)
            infos = [solve_all(handles, mode, A, C) for _ in range(steps)]
            ev1.record(stream)
            barrier()
        finally:
            if clk:
                clk.__exit__(None, None, None)
        for h in handles.values():
            P.pr_set_timing(h, False)
        ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, dist, dev)
        s1 = {p: P.pr_stats(h) for p, h in handles.items()}
        last = infos[-1]
        for p, h in handles.items():
            P.pr_result(h, C)
            last[p]["rel_error_vs_closed_form"] = rel_err(C, p)
        return ms, last, s0, s1, clk

    # ---- the headline: Eq. 3's C_0 (the plain method's start)
    ms, last, s0, s1, clk = timed(arms["eq3"], args.mode, args.steps, args.warmup, sample_clocks=True)
    launches = sum(s1[p]["launches"] - s0[p]["launches"] for p in ps)

    # Roofline of the dominant product kernel over the timed region (CUDA events around every launch).
    def delta(key, k):
        return sum(s1[p][key][k] - s0[p][key][k] for p in ps)

    by_prec = {k: (delta("gemm_ms_by_precision", k), delta("gemm_flops_by_precision", k),
                   delta("gemms_timed_by_precision", k)) for k in range(P.PR_NPREC)}
    dom = max(by_prec, key=lambda k: by_prec[k][0])
    dms, dfl, dn = by_prec[dom]
    peaks, peak_src = load_peaks()
    S = s1[ps[0]]["emu_slices"]
    if dom == P.PR_EMU64:
        pairs = S * (S + 1) // 2
        exec_fl = dfl * pairs
        roofline = {"bound": "tensor", "kernel": "k_gemm_emu (tcgen05 FP16 digit-slice products)",
                    "achieved": exec_fl / (dms * 1e-3) / 1e12, "peak": peaks["bf16_tflops_sustained"],
                    "unit": "TFLOP/s", "traffic": EMU_TRAFFIC_CURRENT.get(args.n) if S == 8 else None,
                    "note": f"algorithmic = the {pairs} FP16 digit-pair products per emulated FP64 product "
                            f"(S={S}), upper-triangle tiles; fp64_equivalent_tflops = FP64 flops / time",
                    "fp64_equivalent_tflops": dfl / (dms * 1e-3) / 1e12,
                    "peak_source": f"{peak_src} bf16 sustained x nominal fp16/bf16 ratio 1 (kernel timed inside a long step)"}
    elif dom in (P.PR_BF16, P.PR_FP8):
        nominal = 2.0 if dom == P.PR_FP8 else 1.0
        roofline = {"bound": "tensor", "kernel": "k_gemm_lowp_tc", "achieved": dfl / (dms * 1e-3) / 1e12,
                    "peak": peaks["bf16_tflops_sustained"] * nominal, "unit": "TFLOP/s", "traffic": None,
                    "peak_source": f"{peak_src} bf16 sustained x nominal ratio {nominal:g}"}
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
        solve_all(arms["eq3"], args.mode, Ah, Ch)
        barrier()
        k = max(1, min(args.steps, args.e2e_steps))
        t0 = time.perf_counter()
        for _ in range(k):
            solve_all(arms["eq3"], args.mode, Ah, Ch)
        barrier()
        nbytes = args.n * args.n * 8 * len(ps)
        e2e = {"value": max_over_ranks((time.perf_counter() - t0) * 1e3 / k, dist, dev), "unit": "ms",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": k}

    def plain_fp64(handles, ref_ms):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(args.compare_warmup):
            solve_all(handles, "fp64", A, C)
        barrier()
        e0.record(stream)
        pinfo = None
        for _ in range(args.compare_steps):
            pinfo = solve_all(handles, "fp64", A, C)
        e1.record(stream)
        barrier()
        for p, h in handles.items():
            P.pr_result(h, C)
            pinfo[p]["rel_error_vs_closed_form"] = rel_err(C, p)
        pms = e0.elapsed_time(e1) / args.compare_steps
        return {"ms_per_step": pms, "speedup_of_value": pms / ref_ms, "steps": args.compare_steps,
                "warmup": args.compare_warmup, "solves": {str(p): v for p, v in pinfo.items()}}

    # ---- the scaled identity C_0 = ||A||_1^{-1/p} I: same solves, FP64-accurate for every p
    si = None
    if "scaled_identity" in arms:
        si_ms, si_last, _, _, _ = timed(arms["scaled_identity"], args.mode, args.steps, args.warmup)
        si = {"ms_per_step": si_ms, "steps": args.steps, "warmup": args.warmup,
              "solves": {str(p): v for p, v in si_last.items()}}

    # ---- the plain FP64 GPU iteration of both starts (the speed comparison)
    plain, plain_si = None, None
    if not args.no_compare and args.mode != "fp64":
        plain = plain_fp64(arms["eq3"], ms)
        if si:
            plain_si = plain_fp64(arms["scaled_identity"], si["ms_per_step"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tot, what = 0.0, []
        for p in ps:
            est, w = oracle_sample(case.A, p, last[p]["iterations"])
            tot += est
            what.append(w)
        what.append("the iteration of Eq. 1 only (the refinement of the p >= 2 roots has no oracle time here)")
        cpu = {"value": tot, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle", "sample": "; ".join(what)}

    for handles in arms.values():
        for h in handles.values():
            P.pr_destroy(h)
    del A, C
    torch.cuda.empty_cache()

    # ---- the other workloads, summarised (their own JSON lines: --workload batched / learned)
    extra = {}
    if not args.no_extra:
        for name, fn in (("batched", measure_batched), ("learned", measure_learned)):
            try:
                sub = fn(args, world, rank, local, dist, args.sub_steps, args.sub_warmup, False, False)
                keep = ("value", "unit", "steps", "warmup", "config", "roofline", "batch", "learned", "plain_eq3",
                        "scaled_identity",
                        "gpu_launches", "clocks")
                extra[name] = {k: sub[k] for k in keep if k in sub}
            except Exception as exc:  # a failing summary must not hide the headline
                extra[name] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()
        try:
            extra["large"] = measure_large(args, local)
        except Exception as exc:
            extra["large"] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()
        try:
            r1 = measure_f1(args, local)
            extra["f1"] = {"ms": r1["value"], "reference_norm": r1["reference_norm"], **r1["table"]}
        except Exception as exc:
            extra["f1"] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()
        try:
            extra["f3"] = measure_f3(args, local)
        except Exception as exc:
            extra["f3"] = {"error": f"{type(exc).__name__}: {exc}"}

    if rank == 0:
        line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fast": "bf16+emu64(fp16 slices)+bf16 refinement solves",
                                               "emu64": "emu64(fp16 slices)",
                                               "fp64": "f64"}[args.mode],
                "data": "synthetic", "config": config_dict(args, ps), "roofline": roofline,
                "kernel_time_share": kernel_share, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "solves": {str(p): v for p, v in last.items()}, "plain_fp64_gpu": plain,
                "scaled_identity": si, "plain_fp64_gpu_scaled_identity": plain_si,
                "ms_per_step_scaled_identity": si["ms_per_step"] if si else None}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
