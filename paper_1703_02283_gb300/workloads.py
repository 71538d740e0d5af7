"""Seeded synthetic inputs for the inverse p-th root solver.

This module builds test and benchmark matrices only. It contains none of the method's arithmetic
(no norms of the method, no initial guess, no iteration, no root), so both the CUDA path and the
CPU oracle may consume what it produces.

Recipes (all seeded with ``numpy.random.default_rng``):

* ``spd_from_spectrum(n, lam_min, seed)``: ``A = Q diag(lam) Q^T`` with ``Q`` the orthogonal factor of
  the QR factorisation of an ``n x n`` standard-normal matrix (column signs fixed so that ``diag(R) > 0``),
  ``lam`` log-uniform in ``[lam_min, 1]`` with both endpoints pinned (``lam[0] = 1``,
  ``lam[n-1] = lam_min``), and ``A`` symmetrised as ``(A + A^T) / 2``. The condition number is therefore
  exactly ``1 / lam_min``. The paper's matrices are SPD (Sec. 1); the known eigendecomposition lets the
  oracle state the exact root.
* ``overlap_points`` / ``overlap_matrix``: an overlap-type SPD matrix ``S_ij = exp(-|r_i - r_j| / ell)``
  for points uniform in a cube, standing in for the H2O overlap matrices of Sec. 4.1 (unit diagonal,
  entries in (0, 1], decaying with distance), which are not available.
* ``spd_from_spectrum_device``: the same recipe built on the GPU by torch, for the order-16384 case.
* ``batched_specs``: sizes, condition numbers and roots of a batch of independent problems.
* ``sparse_overlap(n, density, seed)``: a sparse overlap-type SPD matrix at the densities Sec. 4.1 reports
  for its H2O overlap matrices (25 % at N = 768, 12.4 % at 1536, 6.2 % at 3072, 3.1 % at 6144: the
  nearsightedness of electronic matter). n points uniform in a cube of side ``20 (n / 2048)^(1/3)`` (the
  point density of the dense stand-in), ordered by their first coordinate (so that the non-zeros of a row
  block fall in a band of columns), ``S_ij = exp(-r_ij) w(r_ij / c)`` with the compactly supported Wendland
  function ``w(t) = (1 - t)^4 (4t + 1)`` for t < 1 (0 beyond), positive definite in three dimensions; the
  product of two positive definite kernels is positive definite, and a unit diagonal keeps
  ``lambda_min`` at least that of the exponential kernel's matrix. The cutoff c is the distance that leaves
  the requested fraction of non-zero entries.
* ``symmetric_perturbation(n, seed)``: a symmetric N(0, 1) matrix scaled to unit Frobenius norm, the
  direction of the error planted in an approximate root that the refinement tests start from.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class SpdCase:
    """One synthetic SPD matrix with its known eigendecomposition."""

    A: np.ndarray  # (n, n) float64, symmetric positive definite, row-major
    Q: np.ndarray  # (n, n) float64, orthogonal
    lam: np.ndarray  # (n,) float64 eigenvalues, A = Q diag(lam) Q^T
    seed: int

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def kappa(self) -> float:
        return float(self.lam.max() / self.lam.min())


def log_uniform_spectrum(rng: np.random.Generator, n: int, lam_min: float) -> np.ndarray:
    """Eigenvalues log-uniform in [lam_min, 1]; the first is pinned to 1 and the last to lam_min."""
    lam = np.exp(rng.uniform(math.log(lam_min), 0.0, n))
    if n >= 1:
        lam[0] = 1.0
    if n >= 2:
        lam[-1] = lam_min
    return lam


def haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Orthogonal factor of a QR factorisation of an n x n N(0, 1) matrix, with diag(R) made positive."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def spd_from_spectrum(n: int, lam_min: float, seed: int) -> SpdCase:
    """A = Q diag(lam) Q^T with the recipe described in the module docstring."""
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(rng, n)
    lam = log_uniform_spectrum(rng, n, lam_min)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    return SpdCase(A=np.ascontiguousarray(A), Q=Q, lam=lam, seed=seed)


@dataclass
class DeviceSpdCase:
    """An SPD matrix built on the device, for orders where the host QR takes minutes."""

    A: object  # (n, n) torch.float64 CUDA tensor, symmetric positive definite
    Q: object  # (n, n) torch.float64 CUDA tensor, orthogonal
    lam: np.ndarray  # (n,) float64 eigenvalues (host)
    seed: int


def spd_from_spectrum_device(n: int, lam_min: float, seed: int, device) -> DeviceSpdCase:
    """The ``spd_from_spectrum`` recipe with the normal matrix, its QR factorisation and the product
    ``Q diag(lam) Q^T`` taken on the device by torch (its normal generator seeded with ``seed``,
    cuSOLVER, cuBLAS). The spectrum is the host recipe's, from ``numpy.random.default_rng(seed)``.
    Same distributions as ``spd_from_spectrum``; not the same matrix."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G = torch.randn((n, n), dtype=torch.float64, device=device, generator=g)
    Q, R = torch.linalg.qr(G)
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    del G, R
    Q.mul_(d)
    lam = log_uniform_spectrum(np.random.default_rng(seed), n, lam_min)
    A = (Q * torch.from_numpy(lam).to(device)) @ Q.T
    At = A.T.contiguous()
    A.add_(At).mul_(0.5)
    del At
    return DeviceSpdCase(A=A, Q=Q, lam=lam, seed=seed)


# Non-zero fraction of the overlap matrices of Sec. 4.1 by order (N = 786 and 1572 read as 768 and 1536).
PAPER_OVERLAP_DENSITY = {768: 0.25, 1536: 0.124, 3072: 0.062, 6144: 0.031}


def sparse_overlap(n: int, density: float, seed: int) -> tuple[np.ndarray, float]:
    """The sparse overlap stand-in described in the module docstring: (S, cutoff c)."""
    from scipy.spatial.distance import pdist, squareform

    box = 20.0 * (n / 2048.0) ** (1.0 / 3.0)
    r = np.random.default_rng(seed).uniform(0.0, box, size=(n, 3))
    r = r[np.argsort(r[:, 0], kind="stable")]
    dist = pdist(r)  # the n (n - 1) / 2 distances of distinct pairs
    pairs = int(round((density * n * n - n) / 2.0))
    pairs = min(max(pairs, 0), dist.size - 1)
    c = float(np.partition(dist, pairs)[pairs])  # the (pairs + 1)-th smallest distance: pairs of them are < c
    near = dist < c
    d = dist[near]
    t = d / c
    u = 1.0 - t
    vals = np.zeros_like(dist)
    vals[near] = np.exp(-d) * (u * u) * (u * u) * (4.0 * t + 1.0)
    S = squareform(vals)
    np.fill_diagonal(S, 1.0)
    return np.ascontiguousarray(S), c


def symmetric_perturbation(n: int, seed: int) -> np.ndarray:
    """(G + G^T) / 2 for an n x n N(0, 1) matrix G, scaled to unit Frobenius norm (a perturbation direction
    with no relation to any matrix's eigenvectors)."""
    G = np.random.default_rng(seed).standard_normal((n, n))
    E = 0.5 * (G + G.T)
    return np.ascontiguousarray(E / np.linalg.norm(E))


# The fixed workloads. Sizes and spectra follow the benchmark recipes: a small plain-FP64 case that the
# oracle finishes in seconds, a single large matrix at kappa = 1e3 for p = 1..4, and a very large one.
SMALL_CASE = dict(n=256, lam_min=1e-2, seed=0, p=2)
SINGLE_CASE = dict(n=4096, lam_min=1e-3, seed=1, p_values=(1, 2, 3, 4))
LARGE_CASE = dict(n=16384, lam_min=1e-4, seed=2, p=2)


def overlap_points(n_points: int, box: float, seed: int) -> np.ndarray:
    """n_points positions uniform in the cube [0, box]^3 (the overlap stand-in's basis-function centres)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, box, size=(n_points, 3))


def jitter_points(r: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """One drift step of a sequence: every coordinate moves by N(0, sigma^2); no wrap-around."""
    return r + rng.normal(0.0, sigma, size=r.shape)


def overlap_matrix(r: np.ndarray, ell: float = 1.0) -> np.ndarray:
    """S_ij = exp(-|r_i - r_j| / ell): symmetric, unit diagonal, positive definite for distinct points."""
    d2 = np.zeros((r.shape[0], r.shape[0]))
    for k in range(r.shape[1]):  # one coordinate at a time: no n x n x 3 temporary
        d2 += (r[:, k, None] - r[None, :, k]) ** 2
    S = np.exp(-np.sqrt(d2) / ell)
    return np.ascontiguousarray(0.5 * (S + S.T))


@dataclass
class BatchSpec:
    n: np.ndarray  # (count,) int sizes
    lam_min: np.ndarray  # (count,) 1/kappa
    p: np.ndarray  # (count,) roots
    seeds: np.ndarray  # (count,) per-matrix seeds


def batched_specs(count: int = 512, n_lo: int = 64, n_hi: int = 1024, kappa_lo: float = 10.0,
                  kappa_hi: float = 1e4, p_choices=(1, 2, 3), seed: int = 999) -> BatchSpec:
    """Sizes uniform in {n_lo..n_hi}, kappa log-uniform in [kappa_lo, kappa_hi], p uniform in p_choices.

    Matrix i is then built by ``spd_from_spectrum(n[i], lam_min[i], seeds[i])`` with seeds 1000 + i.
    """
    rng = np.random.default_rng(seed)
    n = rng.integers(n_lo, n_hi + 1, size=count)
    kappa = np.exp(rng.uniform(math.log(kappa_lo), math.log(kappa_hi), size=count))
    p = rng.choice(np.asarray(p_choices), size=count)
    return BatchSpec(n=n.astype(np.int64), lam_min=1.0 / kappa, p=p.astype(np.int64),
                     seeds=1000 + np.arange(count, dtype=np.int64))
