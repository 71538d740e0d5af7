"""The learned polynomial initial guess: data, training and use of the device MLP (pr_mlp_*).

For a family of slowly drifting SPD matrices (overlap matrices of moving points, the stand-in for the
overlap matrices of Sec. 4.1) a network maps spectral features of A (pr_features: tr(Ahat^k)/n for
k = 1..6, ||A||_1, ||A||_inf) to the coefficients c of a cubic q with C_0 = ||A||_1^{-1/p} q(A/||A||_1)
(PR_C0_POLY). Training targets come from the plain method: its converged root C gives the extreme
eigenvalues of Ahat (lambda_min = ||C||_2^{-p}, lambda_max = ||A||_2, both by power iteration), and the target
is the cubic that makes q(x)^p x closest to 1 in least squares over that interval (x^{1/p}-weighted
basis), i.e. C_0^p A close to I. The library gates every predicted guess against Eq. 2 and falls back to
Eq. 3, so a poor prediction costs iterations, not correctness.

Everything numerical in the solve runs in the library, and so do the label's spectral estimates
(pr_spectral_bounds: power iterations on A and on the converged root, on the device). This module prepares
data (seeded positions) and drives training; the one host computation is the label's least-squares fit of
4 coefficients on 400 points of the spectral interval (training-data tooling, not part of a solve).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import pthroot as P
from . import workloads as W


def box_for(n: int) -> float:
    """Cube side giving the point density of n = 2048 points in a cube of side 20 (lengths in units of l)."""
    return 20.0 * (n / 2048.0) ** (1.0 / 3.0)


def overlap_sequence(seq: int, steps: int, n: int, every: int = 1, sigma: float = 0.01):
    """Matrices S_t (t = 0, every, 2 every, ...) of sequence `seq`: start points seeded 5000 + seq, then a
    jitter of N(0, sigma^2) per coordinate and step (seeded 9000 + seq)."""
    r = W.overlap_points(n, box_for(n), 5000 + seq)
    rng = np.random.default_rng(9000 + seq)
    out = []
    for t in range(steps):
        if t % every == 0:
            out.append(W.overlap_matrix(r))
        r = W.jitter_points(r, sigma, rng)
    return out


def target_coefficients(s1: float, lam_min: float, lam_max: float, p: int, points: int = 400) -> np.ndarray:
    """Label: the cubic minimising sum_x (1 - q(x) x^{1/p})^2 over log-spaced x on the spectral interval of
    A/||A||_1 (s1 = ||A||_1; lam_min, lam_max from pr_spectral_bounds on the plain method's converged root).
    The top end is widened by 10 % so that q stays positive across the margin the library checks above its
    estimate of ||A||_2."""
    lo, hi = lam_min / s1, min(1.1 * lam_max / s1, 1.0)
    x = np.exp(np.linspace(math.log(lo), math.log(hi), points))
    B = np.stack([x ** (i + 1.0 / p) for i in range(4)], axis=1)
    c, *_ = np.linalg.lstsq(B, np.ones(points), rcond=None)
    return c


@dataclass
class Sample:
    features: np.ndarray  # (8,)
    target: np.ndarray    # (4,)
    iterations: int       # plain method (Eq. 3) iterations


def make_samples(torch, mats, p: int, stream: int = 0, tol: float = 1e-12):
    """Features (library) and targets (from the plain method's converged root) for each matrix."""
    dev = torch.device("cuda")
    out = []
    for S in mats:
        n = S.shape[0]
        A = torch.from_numpy(S).to(dev)
        h = P.pr_init(A, n, p, P.pr_default_options(), stream)
        try:
            f = np.array(P.pr_features(h))
            _, its = P.pr_iterate(h, 100, P.PR_EMU64, tol)
            lam_min, lam_max = P.pr_spectral_bounds(h, 60)
        finally:
            P.pr_destroy(h)
        out.append(Sample(f, target_coefficients(float(f[6]), lam_min, lam_max, p), its))
    return out


def init_params(seed: int) -> np.ndarray:
    """He-initialised parameters (W1 64x8, b1, W2 64x64, b2, W3 4x64, b3), seeded."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((64, 8)) * math.sqrt(2 / 8), np.zeros(64),
             rng.standard_normal((64, 64)) * math.sqrt(2 / 64), np.zeros(64),
             rng.standard_normal((4, 64)) * math.sqrt(1 / 64), np.zeros(4)]
    return np.concatenate([q.ravel() for q in parts]).astype(np.float32)


@dataclass
class Model:
    params: np.ndarray  # raw-feature parameters (normalisation folded into the first layer)
    loss_history: list


def train(samples, steps: int = 400, lr: float = 3e-3, seed: int = 0, stream: int = 0) -> Model:
    """Full-batch Adam on the device MLP. Features are standardised for training; the standardisation is
    then folded into W1 and b1 so that the returned parameters take raw pr_features output."""
    X = np.stack([s.features for s in samples])
    T = np.stack([s.target for s in samples]).astype(np.float32)
    mu, sd = X.mean(0), X.std(0) + 1e-12
    Xn = ((X - mu) / sd).astype(np.float32)
    m = P.pr_mlp_create(init_params(seed), len(samples), stream)
    hist = []
    try:
        for _ in range(steps):
            hist.append(P.pr_mlp_adam_step(m, np.ascontiguousarray(Xn), np.ascontiguousarray(T), len(samples), lr))
        theta = np.empty(P.PR_MLP_PARAMS, dtype=np.float32)
        P.pr_mlp_get_params(m, theta)
    finally:
        P.pr_mlp_destroy(m)
    W1 = theta[:512].reshape(64, 8).astype(np.float64)
    b1 = theta[512:576].astype(np.float64)
    theta[:512] = (W1 / sd).astype(np.float32).ravel()
    theta[512:576] = (b1 - (W1 / sd) @ mu).astype(np.float32)
    return Model(theta, hist)


def predict(model: Model, features: np.ndarray, stream: int = 0) -> np.ndarray:
    """Coefficients predicted by the device MLP for rows of raw features."""
    F = np.ascontiguousarray(np.atleast_2d(features), dtype=np.float32)
    m = P.pr_mlp_create(model.params, F.shape[0], stream)
    try:
        Y = np.empty((F.shape[0], 4), dtype=np.float32)
        P.pr_mlp_forward(m, F, F.shape[0], Y)
    finally:
        P.pr_mlp_destroy(m)
    return Y.astype(np.float64)


def solve_learned(h: int, mlp: int, precision=P.PR_EMU64, tol: float = 1e-12, max_iter: int = 100):
    """On a handle with A loaded (pr_init or pr_load): features -> network -> gated polynomial C_0 ->
    iterations. Returns (status, iterations, guess used, gate estimate)."""
    f = np.asarray(P.pr_features(h), dtype=np.float32)[None]
    y = np.empty((1, 4), dtype=np.float32)
    P.pr_mlp_forward(mlp, f, 1, y)
    P.pr_set_initial_guess(h, P.PR_C0_POLY, y[0].astype(np.float64))
    st, its = P.pr_iterate(h, max_iter, precision, tol)
    s = P.pr_stats(h)
    return st, its, s["c0"], s["c0_gate"]


def solve_with_guess(torch, S: np.ndarray, p: int, coef, precision=P.PR_EMU64, tol: float = 1e-12, stream: int = 0):
    """One solve from the gated polynomial guess; returns (C, iterations, guess used, gate estimate)."""
    dev = torch.device("cuda")
    o = P.pr_default_options()
    o.c0 = P.PR_C0_POLY
    for i in range(4):
        o.c0_coef[i] = float(coef[i])
    A = torch.from_numpy(S).to(dev)
    h = P.pr_init(A, S.shape[0], p, o, stream)
    try:
        _, its = P.pr_iterate(h, 100, precision, tol)
        st = P.pr_stats(h)
        C = torch.empty_like(A)
        P.pr_result(h, C)
    finally:
        P.pr_destroy(h)
    return C.cpu().numpy(), its, st["c0"], st["c0_gate"]
