"""Pins for the oracle's Newton refinement (the step Sec. 3 and Sec. 5 rely on to turn an approximate root
into a precise one). Each test ties it to something other than its own code: the scalar Newton step for
x^p a = 1, the eigenbasis of a commuting iterate, central differences of the balanced residual, the closed
form root, and the coupled form's known failure to remove non-commuting errors. Planted mistakes in the
linearised operator must fail them.
"""
import numpy as np
import pytest

from oracle import pthroot_oracle as O
from paper_1703_02283_gb300 import workloads as W


def _commuting_pair(n, p, seed):
    """A = Q diag(lam) Q^T and a commuting X = Q diag(x) Q^T that is not the root (x off by up to 20 %)."""
    rng = np.random.default_rng(seed)
    Q = W.haar_orthogonal(rng, n)
    lam = np.exp(rng.uniform(np.log(0.05), 0.0, n))
    x = lam ** (-1.0 / p) * (1.0 + 0.2 * rng.uniform(-1.0, 1.0, n))
    A = O.symmetrize((Q * lam) @ Q.T)
    X = O.symmetrize((Q * x) @ Q.T)
    return A, X, Q, lam, x


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_diagonal_refinement_is_the_scalar_newton_step(p):
    # Diagonal A and X commute and stay diagonal; every diagonal entry then follows Newton's method for
    # f(x) = x^p a - 1, x' = x - f(x) / f'(x) = x + (1 - x^p a) / (p x^(p-1) a). Four distinct entries: the
    # conjugate-gradient solve is exact after at most four iterations.
    a = np.array([0.3, 1.7, 4.0, 9.5])
    x = a ** (-1.0 / p) * np.array([1.05, 0.97, 1.02, 1.04])
    X1, info = O.refine_newton(np.diag(a), np.diag(x), p, max_steps=1, tol=0.0, cg_max=10, cg_tol=1e-15)
    want = x + (1.0 - x ** p * a) / (p * x ** (p - 1) * a)
    np.testing.assert_allclose(np.diag(X1), want, rtol=1e-14, atol=0)
    assert np.count_nonzero(X1 - np.diag(np.diag(X1))) == 0
    assert info.steps == 1 and info.stop in ("max_steps", "tol")  # p = 1: the equation is linear, one step is exact
    # the residual of the balanced form on diagonals is 1 - x^p a, entry by entry
    assert info.residuals[0] == pytest.approx(np.linalg.norm(1.0 - x ** p * a), rel=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_balanced_residual_in_the_eigenbasis(p):
    A, X, Q, lam, x = _commuting_pair(10, p, 40 + p)
    G = O.refine_residual(X, A, p)
    np.testing.assert_allclose(G, (Q * (1.0 - x ** p * lam)) @ Q.T, atol=1e-13)
    Z = (Q * lam ** (-1.0 / p)) @ Q.T
    assert np.linalg.norm(O.refine_residual(Z, A, p)) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_operator_is_the_derivative_of_the_balanced_residual(p):
    # Central differences of X -> -G(X) = sym(X^m A X^m') - I along a symmetric direction, at a point X
    # that does not commute with A.
    case = W.spd_from_spectrum(9, 0.1, 31)
    A = case.A
    X = O.closed_form_root(case.Q, case.lam, p) + 0.05 * W.symmetric_perturbation(9, 32)
    D = W.symmetric_perturbation(9, 33)
    h = 1e-5
    fd = -(O.refine_residual(X + h * D, A, p) - O.refine_residual(X - h * D, A, p)) / (2 * h)
    L = O.refine_operator(X, A, p, D)
    assert np.linalg.norm(L - fd) <= 1e-8 * np.linalg.norm(L)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_correction_equals_the_eigenbasis_solution(p):
    # For X = Q diag(x) Q^T commuting with A = Q diag(lam) Q^T, L_X acts on the eigenbasis entry (a, b) of D
    # as a multiplication by l_ab = [s_m (lam_a x_a^m' + lam_b x_b^m') + s_m' (lam_a x_a^m + lam_b x_b^m)] / 2,
    # s_k = sum_{j<k} x_a^j x_b^(k-1-j) (the first-order change of X^k). So D = Q (G_hat / l) Q^T.
    n = 12
    A, X, Q, lam, x = _commuting_pair(n, p, 50 + p)
    G = W.symmetric_perturbation(n, 60 + p)
    m, mq = p // 2, p - p // 2

    def s(k):
        xa, xb = x[:, None], x[None, :]
        return sum(xa ** j * xb ** (k - 1 - j) for j in range(k)) if k else np.zeros((n, n))

    la, lb = lam[:, None], lam[None, :]
    xa, xb = x[:, None], x[None, :]
    ell = 0.5 * (s(m) * (la * xa ** mq + lb * xb ** mq) + s(mq) * (la * xa ** m + lb * xb ** m))
    want = Q @ ((Q.T @ G @ Q) / ell) @ Q.T
    D, its = O.refine_correction(X, A, p, G, cg_max=400, cg_tol=1e-14)
    assert np.linalg.norm(D - want) <= 1e-10 * np.linalg.norm(want)
    assert its <= 400


@pytest.mark.parametrize("p", [2, 3, 4])
def test_refinement_removes_a_non_commuting_error_quadratically(p):
    # A root with an error that does not commute with A: Newton steps reach the closed form, with the error
    # squared (times a modest constant) at each step; the coupled form of Eq. 1 started from the same
    # iterate keeps the error (it converges to X_0 (X_0^p A)^{-1/p}, not to A^{-1/p}).
    case = W.spd_from_spectrum(64, 1e-2, 5)
    A = case.A
    Z = O.closed_form_root(case.Q, case.lam, p)
    X0 = Z + 1e-3 * np.linalg.norm(Z) * W.symmetric_perturbation(64, 11)
    errs = [O.forward_error(X0, Z)]
    X = X0
    for _ in range(3):
        X, info = O.refine_newton(A, X, p, max_steps=1, tol=0.0)
        assert info.steps == 1
        errs.append(O.forward_error(X, Z))
    assert errs[1] < 1e-2 * errs[0] and errs[2] < 1e-4 * errs[1]
    assert errs[2] <= 100.0 * errs[1] ** 2
    assert errs[3] < 1e-14
    Xc, Mc = O.coupled_start(X0, A, p)
    for _ in range(40):
        Xc, Mc = O.step_coupled(Xc, Mc, p)
    assert np.linalg.norm(np.eye(64) - Mc) < 1e-12  # the coupled form "converged"...
    assert O.forward_error(Xc, Z) > 1e-4             # ...to the wrong matrix


def test_refinement_from_eq3_solves_reaches_fp64_accuracy():
    # The coupled form from Eq. 3's C_0 loses accuracy (its M_0 spans kappa^(p+1)); refinement recovers it.
    case = W.spd_from_spectrum(160, 1e-3, 8)
    for p in (2, 3, 4):
        Z = O.closed_form_root(case.Q, case.lam, p)
        C, _ = O.solve(case.A, p, tol=1e-12)
        before = O.forward_error(C, Z)
        X, info = O.refine_newton(case.A, C, p, max_steps=6, tol=0.0)
        after = O.forward_error(X, Z)
        assert before > 1e-9
        assert after < 1e-13, (p, before, after, info)
        assert info.stop == "stagnation" and info.true_residual < 1e-11


def test_stop_rule_outcomes():
    case = W.spd_from_spectrum(48, 1e-2, 9)
    A, p = case.A, 2
    Z = O.closed_form_root(case.Q, case.lam, p)
    X, info = O.refine_newton(A, Z, p, tol=1e-10)
    assert info.stop == "tol" and info.steps == 0 and np.array_equal(X, Z)
    X0 = Z + 1e-2 * np.linalg.norm(Z) * W.symmetric_perturbation(48, 3)
    X, info = O.refine_newton(A, X0, p, max_steps=1, tol=0.0)
    assert info.stop == "max_steps" and info.steps == 1 and len(info.residuals) == 2
    X, info = O.refine_newton(A, X0, p, max_steps=30, tol=0.0)
    assert info.stop == "stagnation" and info.steps < 8
    assert len(info.residuals) == info.steps + 1 and len(info.cg_iterations) == info.steps
    # the returned iterate is the one whose residual was recorded last
    assert np.linalg.norm(O.refine_residual(X, A, p)) == pytest.approx(info.residuals[-1], rel=1e-12)
    assert info.true_residual == pytest.approx(O.residual_fro(X, A, p), rel=1e-12)


def test_planted_mistakes_are_caught(monkeypatch):
    good = O.refine_operator

    def drops_second_term(X, A, p, D):
        m, mq = p // 2, p - p // 2
        dm = sum(np.linalg.matrix_power(X, j) @ D @ np.linalg.matrix_power(X, m - 1 - j) for j in range(m))
        return O.symmetrize(dm @ A @ np.linalg.matrix_power(X, mq)) if m else np.zeros_like(X)

    def wrong_split(X, A, p, D):
        return good(X, A, p + 1, D)

    for bad in (drops_second_term, wrong_split):
        monkeypatch.setattr(O, "refine_operator", bad)
        with pytest.raises(AssertionError):
            test_operator_is_the_derivative_of_the_balanced_residual(2)
        with pytest.raises(AssertionError):
            test_correction_equals_the_eigenbasis_solution(3)
        monkeypatch.setattr(O, "refine_operator", good)
    test_operator_is_the_derivative_of_the_balanced_residual(2)
