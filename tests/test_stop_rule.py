"""Host logic of the library: the stop rule pr_iterate applies (a pure host function of the ABI).

For FP64 histories it must agree with the oracle's stop rule; the low-precision arm is checked on
hand-made histories."""
import math

import numpy as np
import pytest

from oracle import pthroot_oracle as O
from paper_1703_02283_gb300 import workloads as W

P = pytest.importorskip("paper_1703_02283_gb300.pthroot")
F64, BF16 = P.PR_FP64, P.PR_BF16
CONTINUE = -1


def rule(hist, prec, tol=1e-12, **opt):
    o = P.pr_default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    return P.pr_stop_rule(hist, prec, tol, o)


def test_basic_outcomes():
    assert rule([3.0], [F64]) == CONTINUE
    assert rule([3.0, 1e-13], [F64, F64]) == P.PR_OK
    assert rule([3.0, math.nan], [F64, F64]) == P.PR_EDIVERGED
    assert rule([3.0, math.inf], [F64, F64]) == P.PR_EDIVERGED
    # armed below stag_below, fails to halve
    assert rule([1e-4, 0.6e-4], [F64, F64]) == P.PR_ESTAGNATED
    assert rule([1e-4, 0.4e-4], [F64, F64]) == CONTINUE
    # not armed: above stag_below
    assert rule([1e-2, 0.9e-2], [F64, F64]) == CONTINUE
    # different precisions are never compared
    assert rule([1e-4, 0.9e-4], [BF16, F64]) == CONTINUE


def test_low_precision_arms():
    # (a) low-precision arm threshold 0.5
    assert rule([0.4, 0.3], [BF16, BF16]) == P.PR_ESTAGNATED
    assert rule([0.4, 0.3], [F64, F64]) == CONTINUE
    # (b) any increase at low precision: a floor above the threshold, or leaving the basin
    h = [16.0, 15.0, 9.0, 4.0, 3.0, 3.1]
    assert rule(h, [BF16] * 6) == P.PR_ESTAGNATED
    assert rule(h, [F64] * 6) == CONTINUE
    assert rule([16.0, 15.9, 15.95], [BF16] * 3) == P.PR_ESTAGNATED
    assert rule([16.0, 15.9, 15.8], [BF16] * 3) == CONTINUE
    # residuals of different precisions are not compared
    assert rule([16.0, 4.0, 16.0], [F64, F64, BF16]) == CONTINUE


def test_agrees_with_oracle_on_fp64_histories():
    c = W.spd_from_spectrum(96, 0.01, 3)
    for p, tol in [(1, 0.0), (2, 1e-12), (2, 0.0), (3, 1e-9)]:
        _, info = O.solve(c.A, p, tol=tol)
        h = info.residuals
        for k in range(1, len(h) + 1):
            got = rule(h[:k], [F64] * k, tol=tol)
            # The pure rule tests the carried residual only: a verified "inaccurate" stop is a PR_OK of the rule
            # (pr_iterate turns it into PR_EINACCURATE after evaluating the true residual).
            want = {"tol": P.PR_OK, "inaccurate": P.PR_OK, "stagnation": P.PR_ESTAGNATED,
                    "diverged": P.PR_EDIVERGED}.get(info.stop)
            if k < len(h):
                assert got == CONTINUE, (p, k)
            elif info.stop != "max_iter":
                assert got == want, (p, k, info.stop)


def test_bad_arguments():
    assert P._lib.pr_stop_rule(None, None, 0, 0.0, None) == P.PR_EINVAL
