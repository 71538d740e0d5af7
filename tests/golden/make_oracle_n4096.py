"""Writes tests/golden/oracle_n4096.json: what the CPU oracle reaches on the order-4096 solves.

Run from the repository root: ``python tests/golden/make_oracle_n4096.py`` (about fifteen minutes on eight
cores). It calls only ``oracle/`` and the seeded input generator; nothing here touches the CUDA path.

Cases:
* the single-matrix recipe, n = 4096, lambda log-uniform in [1e-3, 1], seed 1, p = 1..4, Eq. 3's C_0
  (Newton-Schulz form for p = 1, the coupled form otherwise);
* independent order-4096 instances of the large recipe (lambda in [1e-4, 1], p = 2, seeds 20 and 21) from
  the scaled identity C_0 = ||A||_1^{-1/2} I that Sec. 2 allows;
* the single-matrix recipe again for p = 1..4 from the scaled identity C_0 = ||A||_1^{-1/p} I. Its M_0
  spans only kappa (not kappa^(p+1) as Eq. 3's does), so the oracle's own forward error stays near 1e-13
  for every p and the GPU results can be held to a bar near 1e-12 at full size.

Per case it stores the oracle's iteration count, stop reason, residual history, true residual
||I - C^p A||_F of its result, relative Frobenius error
against the closed form Q diag(lambda^{-1/p}) Q^T, and a sampled block of the oracle's result at seeded
indices (16 x 16 for the Eq. 3 cases, 64 x 64 for the scaled-identity cases of the single-matrix recipe). The GPU tests compare their own solves with these. The inputs are regenerated on the
machine that runs the tests; LAPACK builds may differ there in the last bits of Q, which moves the
errors by far less than the tolerances the tests derive from them.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pthroot_oracle as O  # noqa: E402
from paper_1703_02283_gb300 import workloads as W  # noqa: E402

TOL = 1e-12
CASES = [dict(n=4096, lam_min=1e-3, seed=1, p=p, c0="eq3") for p in (1, 2, 3, 4)] + [
    dict(n=4096, lam_min=1e-4, seed=s, p=2, c0="scaled_identity") for s in (20, 21)] + [
    dict(n=4096, lam_min=1e-3, seed=1, p=p, c0="scaled_identity", block=64) for p in (1, 2, 3, 4)]


def block_indices(n: int, seed: int, k: int = 16) -> np.ndarray:
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def main() -> None:
    out = {"description": __doc__.split("\n\n")[0], "tol": TOL, "cases": []}
    cache = {}
    for c in CASES:
        key = (c["n"], c["lam_min"], c["seed"])
        if key not in cache:
            cache = {key: W.spd_from_spectrum(*key)}
        case = cache[key]
        C, info = O.solve(case.A, c["p"], c0=c["c0"], tol=TOL)
        Z = O.closed_form_root(case.Q, case.lam, c["p"])
        k = c.pop("block", 16)
        idx = block_indices(c["n"], 7000 + c["seed"] * 10 + c["p"] + (0 if k == 16 else 500), k)
        rec = dict(c, form=info.form, iterations=info.iterations, stop=info.stop,
                   residuals=[float(r) for r in info.residuals], forward_error=O.forward_error(C, Z),
                   true_residual=O.residual_fro(C, case.A, c["p"]),
                   block_indices=[int(i) for i in idx], block=C[np.ix_(idx, idx)].tolist(),
                   seconds=round(info.seconds, 1))
        out["cases"].append(rec)
        print(f"n={c['n']} lam_min={c['lam_min']:g} seed={c['seed']} p={c['p']} c0={c['c0']}: "
              f"{info.iterations} it ({info.stop}), r={info.residuals[-1]:.2e}, "
              f"true={rec['true_residual']:.2e}, fwd={rec['forward_error']:.2e}, {info.seconds:.0f} s", flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_n4096.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
