"""Pins of the oracle's custom-precision simulation (the paper's experiment of Sec. 4.3, Fig. 2): the
mantissa rounding against IEEE half and single precision, a product in 2-bit arithmetic worked by hand, the
limits m -> 52 (FP64 itself), and the iteration's behaviour in both modes on a small overlap matrix."""
import numpy as np
import pytest

from oracle import pthroot_oracle as O
from paper_1703_02283_gb300 import workloads as W


def test_round_mantissa_is_half_and_single_precision():
    # m = 10 and m = 23 are the stored mantissas of IEEE half and single precision: within their normal ranges
    # the rounding equals numpy's conversions (one rounding from FP64, ties to even).
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-8, 8, 20000))
    ties = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -(1 + 5 * 2.0 ** -11), 1024 + 0.5, 3 * 2.0 ** -12])
    for v in (x, ties):
        h = v[(np.abs(v) > 2.0 ** -14) & (np.abs(v) < 60000)]
        np.testing.assert_array_equal(O.round_mantissa(h, 10), h.astype(np.float16).astype(np.float64))
        s = v[(np.abs(v) > 2.0 ** -126)]
        np.testing.assert_array_equal(O.round_mantissa(s, 23), s.astype(np.float32).astype(np.float64))
    assert O.round_mantissa(1 + 2.0 ** -11, 10) == 1.0 and O.round_mantissa(1 + 3 * 2.0 ** -11, 10) == 1 + 2.0 ** -9
    assert O.round_mantissa(0.0, 4) == 0.0 and O.round_mantissa(-3.0, 1) == -3.0 and O.round_mantissa(7.0, 1) == 8.0
    np.testing.assert_array_equal(O.round_mantissa(x, 52), x)


def test_matmul_rounded_by_hand():
    # m = 2 (3 significant bits): 1.5 x 1.25 = 1.875 is a tie between 1.75 and 2 -> 2 (even);
    # 1.25 x 1.75 = 2.1875 -> 2; 2 + 2 = 4. A second column: 1.5 x 1 = 1.5, 1.25 x 3 = 3.75 -> 4 (tie -> even
    # 4), 1.5 + 4 = 5.5 -> 6 (tie between 5 and 6 -> 6).
    X = np.array([[1.5, 1.25]])
    Y = np.array([[1.25, 1.0], [1.75, 3.0]])
    np.testing.assert_array_equal(O.matmul_rounded(X, Y, 2), np.array([[4.0, 6.0]]))
    # m = 52: FP64 itself, summed in order k = 0, 1, ...
    rng = np.random.default_rng(1)
    A, B = rng.standard_normal((7, 9)), rng.standard_normal((9, 5))
    want = np.zeros((7, 5))
    for k in range(9):
        want = want + np.outer(A[:, k], B[k, :])
    np.testing.assert_array_equal(O.matmul_rounded(A, B, 52), want)


def test_quantized_iterates_limits_and_modes():
    # An overlap matrix of 40 points (unit diagonal, kappa ~ 14): with m = 52 storage is the literal FP64
    # iteration exactly, and arithmetic (another summation order) agrees with it to rounding until the root
    # is reached (iteration 18); after that the literal order amplifies rounding by about 3 per iteration in
    # both. Storage with few bits still converges to its floor; arithmetic needs more bits.
    r = W.overlap_points(40, 20.0 * (40 / 2048) ** (1 / 3), 3)
    S = W.overlap_matrix(r)
    Z = O.eig_root(S, 2)
    Cs = O.quantized_iterates(S, 2, 52, "storage", 25)
    Ca = O.quantized_iterates(S, 2, 52, "arithmetic", 25)
    lit = O.initial_guess_eq3(S)
    for k in range(26):
        assert np.array_equal(Cs[k], lit), k
        if k <= 18:
            assert O.forward_error(Ca[k], lit) < 1e-14, k
        lit = O.step_literal(lit, S, 2)
    assert min(O.forward_error(C, Z) for C in Cs) < 1e-14
    # Few bits: the error first falls as in FP64, down to a floor set by the precision (the first phase of
    # Sec. 4.3), then the literal order amplifies the rounding and the error grows again (the paper saw
    # oscillations there). The floor: about the stored rounding for storage, more for arithmetic.
    def floor(m, mode):
        with np.errstate(over="ignore", invalid="ignore"):
            e = [O.forward_error(C, Z) for C in O.quantized_iterates(S, 2, m, mode, 25)]
        return np.nanmin(np.asarray(e))
    assert floor(4, "storage") < 0.1 and floor(16, "storage") < 1e-4
    assert floor(16, "arithmetic") < 1e-3 and floor(4, "arithmetic") > floor(4, "storage")
