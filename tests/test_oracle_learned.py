"""Pins for the oracle's learned-initial-guess functions: spectral features, the polynomial C_0, the
Eq. 2 gate, the relative least-squares fit, and the MLP's forward pass and gradient."""
import numpy as np
import pytest

from oracle import pthroot_oracle as O
from paper_1703_02283_gb300 import workloads as W


def test_features_closed_form():
    c = W.spd_from_spectrum(40, 0.05, 3)
    f = O.spectral_features(c.A)
    s = O.norm_1(c.A)
    want = [np.sum((c.lam / s) ** k) / 40 for k in range(1, 7)]  # traces from the known eigenvalues
    np.testing.assert_allclose(f[:6], want, rtol=1e-12)
    assert f[6] == O.norm_1(c.A) and f[7] == O.norm_inf(c.A)


def test_polynomial_guess_eigenvalues_and_special_cases():
    c = W.spd_from_spectrum(30, 0.1, 4)
    s = O.norm_1(c.A)
    coef = [0.7, -0.2, 0.4, 0.1]
    C0 = O.polynomial_initial_guess(c.A, 2, coef)
    x = c.lam / s
    q = coef[0] + coef[1] * x + coef[2] * x ** 2 + coef[3] * x ** 3
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(C0)), np.sort(s ** -0.5 * q), rtol=1e-12)
    # c = (1, 0, 0, 0) is the scaled identity; c = (0, 1/s... ) reproduces Eq. 3 for p = 1: C_0 = A / s^2
    np.testing.assert_allclose(O.polynomial_initial_guess(c.A, 3, [1, 0, 0, 0]),
                               O.initial_guess_scaled_identity(c.A, 3), rtol=1e-14)
    np.testing.assert_allclose(O.polynomial_initial_guess(c.A, 1, [0, 1, 0, 0]), O.initial_guess_eq3(c.A),
                               rtol=1e-13, atol=1e-16)


def test_gate_matches_scalar_model():
    c = W.spd_from_spectrum(30, 0.1, 5)
    for p in (1, 2, 3):
        C0 = O.initial_guess_eq3(c.A)
        mu = (c.lam / (O.norm_1(c.A) * O.norm_inf(c.A))) ** p * c.lam
        assert O.gate_value(c.A, p, C0) == pytest.approx(np.abs(1 - mu).max(), rel=1e-12)


def test_relative_fit_narrow_interval_and_quality():
    for p in (1, 2, 3):
        a = 0.3
        c = O.relative_fit(a, a * (1 + 1e-6), p)
        q = np.polyval(c[::-1], a)
        assert q * a ** (1.0 / p) == pytest.approx(1.0, abs=1e-6)
        # On a wide interval the fit keeps q(x)^p x in (0, 2): the gate of Eq. 2 holds on the spectrum.
        lo = 1e-2
        c = O.relative_fit(lo, 1.0, p)
        x = np.exp(np.linspace(np.log(lo), 0.0, 2000))
        qx = np.polyval(c[::-1], x)
        assert np.all(qx > 0) and np.abs(1 - qx ** p * x).max() < 1.0


def test_relative_fit_cuts_iterations():
    c = W.spd_from_spectrum(64, 1e-2, 6)
    s = O.norm_1(c.A)
    for p in (1, 2, 3):
        coef = O.relative_fit(c.lam.min() / s, c.lam.max() / s, p)
        C0 = O.polynomial_initial_guess(c.A, p, coef)
        assert O.gate_value(c.A, p, C0) < 0.9
        _, info_poly = O.solve(c.A, p, C0=C0, tol=1e-12)
        _, info_eq3 = O.solve(c.A, p, tol=1e-12)
        Z = O.closed_form_root(c.Q, c.lam, p)
        assert info_poly.iterations < info_eq3.iterations
        assert O.forward_error(O.solve(c.A, p, C0=C0, tol=1e-12)[0], Z) < 1e-12


def test_mlp_hand_case_and_finite_differences():
    rng = np.random.default_rng(0)
    # Hand case: only b3 non-zero -> Y = b3 for every sample; loss = mean (b3 - t)^2; d/db3 = 2 (b3 - t_mean) / 4.
    theta = np.zeros(O.MLP_PARAMS)
    theta[-4:] = [1.0, -2.0, 0.5, 3.0]
    X = rng.standard_normal((5, 8))
    T = rng.standard_normal((5, 4))
    loss, g = O.mlp_loss_grad(theta, X, T)
    np.testing.assert_allclose(O.mlp_forward(theta, X), np.tile(theta[-4:], (5, 1)))
    assert loss == pytest.approx(np.mean((theta[-4:] - T) ** 2))
    np.testing.assert_allclose(g[-4:], 2 * (theta[-4:] - T.mean(0)) / 4, rtol=1e-12)
    # Central differences on a random network (ReLU kinks avoided by the random draw).
    theta = rng.standard_normal(O.MLP_PARAMS) * 0.3
    X = rng.standard_normal((7, 8))
    T = rng.standard_normal((7, 4))
    loss, g = O.mlp_loss_grad(theta, X, T)
    idx = rng.choice(O.MLP_PARAMS, 60, replace=False)
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (O.mlp_loss_grad(tp, X, T)[0] - O.mlp_loss_grad(tm, X, T)[0]) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-9)
