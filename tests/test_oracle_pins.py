"""Pins for the CPU oracle: each test ties it to something other than itself (hand-derived values,
closed forms, LAPACK, the scalar recurrence in the eigenbasis, invariants), so that a plausible
mistake in the oracle (a dropped term, a wrong coefficient, a transposed operand, a wrong product
order) fails at least one of them. ``test_planted_mistakes_are_caught`` checks that claim directly.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import pthroot_oracle as O
from paper_1703_02283_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _case(n, lam_min, seed):
    return W.spd_from_spectrum(n, lam_min, seed)


# ------------------------------------------------------------------------- Eq. 3: norms and C_0

def test_norms_hand_matrix():
    A = np.array([[1.0, -2.0], [3.0, 4.0]])
    # column sums |1|+|3| = 4, |-2|+|4| = 6; row sums 3, 7
    assert O.norm_1(A) == 6.0
    assert O.norm_inf(A) == 7.0
    B = np.random.default_rng(3).standard_normal((7, 5))
    assert O.norm_1(B) == pytest.approx(np.linalg.norm(B, 1), rel=1e-15)
    assert O.norm_inf(B) == pytest.approx(np.linalg.norm(B, np.inf), rel=1e-15)


def test_eq3_initial_guess_is_transpose_over_norm_product():
    A = np.array([[1.0, -2.0], [3.0, 4.0]])
    C0 = O.initial_guess_eq3(A)
    np.testing.assert_array_equal(C0 * 42.0, np.array([[1.0, 3.0], [-2.0, 4.0]]))


def test_eq2_holds_for_eq3_guess_exactly_from_spectrum():
    # C_0 = A/s with s = ||A||_1 ||A||_inf; eigenvalues of C_0^p A are lam^{p+1}/s^p.
    for (n, lam_min, seed) in [(64, 1e-2, 0), (128, 1e-3, 1)]:
        c = _case(n, lam_min, seed)
        s = O.norm_1(c.A) * O.norm_inf(c.A)
        for p in (1, 2, 3, 4):
            mu = c.lam ** (p + 1) / s ** p
            assert np.all(mu > 0) and np.all(mu < 1)
            C0 = O.initial_guess_eq3(c.A)
            E = np.eye(n) - np.linalg.matrix_power(C0, p) @ c.A
            # 1 - mu_min may round to 1 in FP64 (mu_min ~ kappa^-(p+1)); the strict bound is on mu.
            assert np.linalg.norm(E, 2) == pytest.approx(1.0 - mu.min(), rel=1e-12)
            assert np.linalg.norm(E, 2) <= 1.0


def test_eq2_scaling_caveat_small_norm():
    # Reading: for p > 1 the guess of Eq. 3 is not scale-invariant; A = 0.1 I, p = 2 gives C_0^2 A = 10 I.
    A = 0.1 * np.eye(3)
    C0 = O.initial_guess_eq3(A)
    assert np.linalg.norm(np.eye(3) - C0 @ C0 @ A, 2) == pytest.approx(9.0, rel=1e-12)


def test_eq2_prescale_restores_convergence():
    # A = 0.1 I, p = 2: Eq. 3 on A itself diverges; on 2^k A (||2^k A||_1 = 1.6) Eq. 2 holds exactly
    # (from the spectrum) and 2^(k/2) times the limit is 0.1^(-1/2) I.
    A = 0.1 * np.eye(4)
    _, info = O.solve(A, 2, tol=1e-14, max_iter=40)
    assert info.stop == "diverged" or info.residuals[-1] > 1.0
    As, k = O.eq2_prescale(A, 2)
    assert k == 4 and np.array_equal(As, 1.6 * np.eye(4)) and 1.0 <= O.norm_1(As) < 2.0
    mu = 1.6 ** 3 / (O.norm_1(As) * O.norm_inf(As)) ** 2  # eigenvalue of C_0^2 As
    assert abs(1.0 - mu) < 1.0
    C, info = O.solve(As, 2, tol=1e-14)
    assert info.stop in ("tol", "stagnation")
    np.testing.assert_allclose(2.0 ** (k / 2) * C, 0.1 ** -0.5 * np.eye(4), rtol=1e-14)


@pytest.mark.parametrize("p", [2, 3])
def test_eq2_prescale_matches_closed_form(p):
    # A random SPD matrix shrunk below ||A||_1 = 1: the scaled solve, scaled back, is the closed-form root of
    # the shrunk matrix; k = 0 when nothing needs scaling (p = 1, or ||A||_1 >= 1).
    c = _case(40, 0.05, 21)
    A = 0.01 * c.A
    As, k = O.eq2_prescale(A, p)
    assert k > 0 and 1.0 <= O.norm_1(As) < 2.0 and np.array_equal(As, A * 2.0 ** k)
    C, info = O.solve(As, p, tol=1e-13)
    Z = O.closed_form_root(c.Q, 0.01 * c.lam, p)
    # Eq. 3's M_0 spans kappa^(p+1) = 20^4: about u kappa^(p+1) = 3.6e-11 of relative error is carried.
    assert O.forward_error(2.0 ** (k / p) * C, Z) < 1e-11
    assert O.eq2_prescale(A, 1)[1] == 0 and O.eq2_prescale(c.A, p)[1] == 0


# ------------------------------------------------------------------------- hand-derived iterates

def _golden_cases():
    with open(os.path.join(GOLDEN, "dyadic_iterates.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: f"p{c['p']}-n{len(c['A_diag'])}")
def test_golden_dyadic_iterates(case):
    A = np.diag(np.array(case["A_diag"]))
    p = case["p"]
    want = [np.diag([float(Fraction(v)) for v in it]) for it in case["iterates"]]
    forms = ["literal", "coupled"] + (["ns"] if p == 1 else [])
    for form in forms:
        for k, W_k in enumerate(want):
            C, info = O.solve(A, p, form=form, c0="eq3", tol=0.0, max_iter=k, stag_below=0.0)
            assert info.iterations == k
            np.testing.assert_array_equal(C, W_k, err_msg=f"form={form} k={k}")


def test_golden_scalar_recurrence_exact_rationals():
    # The scalar recurrence itself against exact rational arithmetic.
    lam = np.array([4.0])
    c = O.scalar_recurrence(lam, np.array([0.25]), 2, 2)
    assert c[0] == float(Fraction(7117, 16384))


# ------------------------------------------------------------------------- limits: closed forms

@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_limit_matches_closed_form_and_lapack(p):
    c = _case(48, 1e-1, 11)
    Z = O.closed_form_root(c.Q, c.lam, p)
    Ze = O.eig_root(c.A, p)
    assert O.forward_error(Ze, Z) < 1e-13
    for c0 in ("eq3", "scaled_identity"):
        C, info = O.solve(c.A, p, c0=c0, tol=1e-13)
        assert info.stop in ("tol", "stagnation", "inaccurate")
        assert O.forward_error(C, Z) < 1e-12, (c0, info)
        # Z^p A = I (definition of the inverse p-th root)
        assert O.residual_fro(Z, c.A, p) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_closed_form_block_and_residual_rows(p):
    # Entry-wise closed form: on every row pair it is an inverse p-th root (Z^p A = I, Z symmetric) and
    # the inverse itself for p = 1; a block of it is the same block of the full root.
    c = _case(40, 5e-2, 13)
    Z = O.closed_form_block(c.Q, c.Q, c.lam, p)
    assert np.linalg.norm(np.linalg.matrix_power(Z, p) @ c.A - np.eye(40)) < 1e-11
    assert np.array_equal(Z, Z.T) or np.abs(Z - Z.T).max() < 1e-13
    if p == 1:
        np.testing.assert_allclose(Z, np.linalg.inv(c.A), rtol=1e-11, atol=1e-12)
    rows, cols = np.array([3, 17, 39]), np.array([0, 17, 22, 5])
    np.testing.assert_allclose(O.closed_form_block(c.Q[rows], c.Q[cols], c.lam, p), Z[np.ix_(rows, cols)],
                               rtol=1e-13, atol=1e-15)
    # Residual rows: zero (to rounding) at the root, e_i - (row i of C^p) A in general, here for C = A
    # (rows of I - A^{p+1}, formed independently by matrix_power).
    assert np.abs(O.residual_rows(Z, c.A, p, rows)).max() < 1e-12
    want = (np.eye(40) - np.linalg.matrix_power(c.A, p + 1))[rows]
    np.testing.assert_allclose(O.residual_rows(c.A, c.A, p, rows), want, rtol=1e-12, atol=1e-14)


def test_p1_is_the_inverse():
    c = _case(64, 1e-2, 5)
    C, info = O.solve(c.A, 1, tol=1e-13)
    assert info.form == "ns"
    Ainv = np.linalg.inv(c.A)
    assert np.linalg.norm(C - Ainv) / np.linalg.norm(Ainv) < 1e-13
    assert np.linalg.norm(C @ c.A - np.eye(64)) < 1e-12


@pytest.mark.parametrize("n", [3, 5, 8])
def test_brute_force_tiny_random_spd(n):
    # Not built from a known eigendecomposition: a random SPD matrix, root from LAPACK.
    rng = np.random.default_rng(100 + n)
    G = rng.standard_normal((n, n))
    A = G @ G.T + 0.5 * np.eye(n)
    for p in (1, 2, 3):
        Z = O.eig_root(A, p)
        C, info = O.solve(A, p, c0="scaled_identity", tol=1e-14)
        assert O.forward_error(C, Z) < 1e-12
        assert np.linalg.norm(np.linalg.matrix_power(Z, p) @ A - np.eye(n)) < 1e-11


# ------------------------------------------------------------------------- every iterate: scalar recurrence

@pytest.mark.parametrize("form,p", [("ns", 1), ("coupled", 1), ("coupled", 2), ("coupled", 3),
                                    ("coupled", 4), ("literal", 1), ("literal", 2), ("literal", 3)])
def test_residual_history_matches_scalar_recurrence(form, p):
    # In the eigenbasis Eq. 1 is c' = ((p+1)c - c^{p+1} lam)/p per eigenvalue, so in exact arithmetic
    # ||I - C_k^p A||_F = sqrt(sum (1 - c_k^p lam)^2) at every k. Compare while well above roundoff.
    c = _case(96, 0.1, 21)
    s = O.norm_1(c.A) * O.norm_inf(c.A)
    C, info = O.solve(c.A, p, form=form, c0="eq3", tol=1e-9, max_iter=60, stag_below=0.0)
    want = O.scalar_residuals(c.lam, c.lam / s, p, len(info.residuals) - 1)
    got = np.asarray(info.residuals)
    mask = want > 1e-6
    assert mask.sum() >= 5
    np.testing.assert_allclose(got[mask], want[mask], rtol=1e-8)
    assert info.iterations == len(info.residuals) - 1


def test_iterations_grow_with_p():
    # Sec. 4.3: more iterations as p grows (scalar recurrence and oracle agree on the counts).
    c = _case(128, 1e-2, 4)
    its = [O.solve(c.A, p, c0="eq3", tol=1e-10)[1].iterations for p in (1, 2, 3, 4)]
    assert its == sorted(its) and its[0] < its[-1]


def test_quadratic_tail():
    # Near convergence each eigencomponent obeys 1 - m' = 1 - (1 - e)(1 + e/p)^p ~ (p+1)/(2p) e^2.
    c = _case(64, 0.1, 8)
    for p in (1, 2, 3):
        C, info = O.solve(c.A, p, c0="scaled_identity", tol=1e-14)
        r = np.asarray(info.residuals)
        tail = [(r[k], r[k + 1]) for k in range(len(r) - 1) if 1e-6 < r[k] < 1e-2]
        assert tail, r
        for a, b in tail:
            assert b <= 4.0 * (p + 1) / (2 * p) * a * a + 1e-13


# ------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("form,p", [("ns", 1), ("coupled", 2), ("coupled", 3), ("literal", 2)])
def test_symmetry_and_commutation(form, p):
    c = _case(64, 0.05, 9)
    for k in (1, 4, 9):
        C, _ = O.solve(c.A, p, form=form, c0="eq3", tol=0.0, max_iter=k, stag_below=0.0)
        assert np.array_equal(C, C.T)
        comm = np.linalg.norm(C @ c.A - c.A @ C) / (np.linalg.norm(C) * np.linalg.norm(c.A))
        assert comm < 1e-13


def test_forms_agree_well_conditioned():
    c = _case(64, 0.2, 2)
    for p in (1, 2, 3):
        Cs = [O.solve(c.A, p, form=f, c0="eq3", tol=0.0, max_iter=8, stag_below=0.0)[0]
              for f in (["literal", "coupled"] + (["ns"] if p == 1 else []))]
        for C in Cs[1:]:
            assert O.forward_error(C, Cs[0]) < 1e-12


# ------------------------------------------------------------------------- stop rule

def test_stop_rule_outcomes():
    c = _case(32, 0.1, 1)
    C, info = O.solve(c.A, 2, tol=1e-8)
    assert info.stop == "tol" and info.residuals[-1] <= 1e-8 and info.residuals[-2] > 1e-8
    assert info.true_residual == O.residual_fro(C, c.A, 2) <= 1e-8
    _, info = O.solve(c.A, 2, tol=0.0, max_iter=3, stag_below=0.0)
    assert info.stop == "max_iter" and info.iterations == 3 and len(info.residuals) == 4
    _, info = O.solve(c.A, 1, tol=0.0)  # the floor cannot be passed: stagnation
    assert info.stop == "stagnation" and info.residuals[-2] < 1e-3
    bad = c.A.copy()
    bad[0, 0] = np.nan
    _, info = O.solve(bad, 2, tol=1e-8)
    assert info.stop == "diverged"


def test_verified_stop_of_the_coupled_form():
    # Eq. 3's M_0 spans kappa^(p+1): at kappa = 1e3, p = 3 the carried ||I - M||_F reaches 1e-12 while the
    # true residual of X stays far above it (rounding carried in M), so the verified stop is "inaccurate";
    # without verification it is "tol". The scaled identity (M_0 spans kappa) meets the same tolerance for
    # real. The Newton-Schulz form tests the true residual itself.
    c = W.spd_from_spectrum(128, 1e-3, 5)
    C, info = O.solve(c.A, 3, tol=1e-12)
    assert info.stop == "inaccurate" and info.residuals[-1] <= 1e-12
    assert info.true_residual == O.residual_fro(C, c.A, 3) > 1e-9
    _, info2 = O.solve(c.A, 3, tol=1e-12, verify=False)
    assert info2.stop == "tol" and info2.true_residual == -1.0
    c = _case(64, 0.1, 5)
    C, info = O.solve(c.A, 3, c0="scaled_identity", tol=1e-12)
    assert info.stop == "tol" and info.true_residual == O.residual_fro(C, c.A, 3) <= 1e-12
    C, info = O.solve(c.A, 1, tol=1e-12)
    assert info.true_residual == info.residuals[-1]


# ------------------------------------------------------------------------- the pins catch mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible mistakes in the oracle's update and check that the scalar-recurrence pin fails."""
    c = _case(48, 0.1, 21)
    s = O.norm_1(c.A) * O.norm_inf(c.A)
    want = O.scalar_residuals(c.lam, c.lam / s, 2, 12)

    def history():
        _, info = O.solve(c.A, 2, form="coupled", c0="eq3", tol=0.0, max_iter=12, stag_below=0.0)
        return np.asarray(info.residuals)

    np.testing.assert_allclose(history(), want, rtol=1e-8)
    good = O.step_coupled

    def wrong_coefficient(X, M, p):
        n = X.shape[0]
        N = (p * np.eye(n) - M) / p  # (p + 1) dropped to p
        Mn = M
        for _ in range(p):
            Mn = O.sym_product(N, Mn)
        return O.sym_product(X, N), Mn

    def missing_power(X, M, p):
        n = X.shape[0]
        N = ((p + 1) * np.eye(n) - M) / p
        return O.sym_product(X, N), O.sym_product(N, M)  # N^p M with one factor only

    for bad in (wrong_coefficient, missing_power):
        monkeypatch.setattr(O, "step_coupled", bad)
        h = history()
        assert not np.allclose(h, want, rtol=1e-6), bad.__name__
        monkeypatch.setattr(O, "step_coupled", good)

    # A transposed, non-symmetric initial guess would break the Eq. 3 hand pin.
    A = np.array([[1.0, -2.0], [3.0, 4.0]])
    assert not np.array_equal(A / 42.0, O.initial_guess_eq3(A))
