"""Plain FP64 CPU oracle for the inverse p-th root iteration (Lass, Kuehne, Plessl, arXiv:1703.02283).

TEST INFRASTRUCTURE ONLY. This module is imported by the tests, by ``__graft_entry__.smoke()`` and by
the benchmark's CPU-baseline leg, and by nothing else. It shares no code with the CUDA path: the only
common input is the seeded matrix generator in ``paper_1703_02283_gb300.workloads``, which holds none of
the method's arithmetic.

What it computes. For a symmetric positive definite ``A`` and an integer ``p >= 1`` the method of Sec. 2
refines an initial guess ``C_0`` by Eq. 1,

    C_{k+1} = ((p + 1) C_k - C_k^{p+1} A) / p,

which converges to ``A^{-1/p}`` when ``||I - C_0^p A||_2 < 1`` (Eq. 2). Eq. 3 gives the initial guess
``C_0 = A^T / (||A||_1 ||A||_inf)``. For p = 1 the iteration is Newton-Schulz for the inverse (Sec. 2).

Forms. Three evaluation orders are provided; all produce the same iterates in exact arithmetic, because
every iterate is a polynomial in ``A`` and therefore commutes with it:

* ``literal``: Eq. 1 exactly as printed, ``C^{p+1} A`` formed right to left (``T = A``, then ``p + 1``
  times ``T = C T``).
* ``ns`` (p = 1 only): ``C (2I - A C)``, the Newton-Schulz form named in Sec. 2.
* ``coupled``: ``X_0 = C_0``, ``M_0 = X_0^p A``; ``N_k = ((p+1) I - M_k) / p``, ``X_{k+1} = X_k N_k``,
  ``M_{k+1} = N_k^p M_k``. Since ``X_{k+1} = X_k ((p+1) I - X_k^p A) / p`` this is Eq. 1 with the product
  ``X_k^p A`` carried along as ``M_k`` instead of being recomputed. (Reading: the literal order is
  numerically unstable for ill-conditioned ``A``, so the coupled order is what the library and this
  oracle run for p >= 2, and ``ns`` for p = 1.)

Readings where the paper is silent. Iterates are kept symmetric, ``(Y + Y^T) / 2``: in the coupled
form every product (its factors commute exactly in exact arithmetic), in the Newton-Schulz and literal
forms only the new iterate (their inner products ``A C`` and ``C^j A`` stay unsymmetrised); the stop
test uses the Frobenius residual ``||I - C^p A||_F`` (the coupled form uses ``||I - M_k||_F``, the same
quantity in exact arithmetic) against a tolerance, with a stagnation exit once the residual is below
``stag_below`` and fails to halve; the error metric is the Frobenius distance to the exact root (Sec. 4.3).

Pins (tests/test_oracle_pins.py): the p = 1 limit equals the matrix inverse; the limit equals the closed
form ``Q diag(lam^{-1/p}) Q^T`` and a LAPACK eigendecomposition root; the per-iteration residual equals
the scalar recurrence of Eq. 1 in the eigenbasis; hand-computed dyadic iterates of small diagonal cases
(tests/golden); the Eq. 2 bound for Eq. 3's guess; symmetry and commutation invariants; the three forms
agree; the quadratic tail.

Learned initial guess (the functions after ``forward_error``): spectral features ``tr(Ahat^k)/n``
(``Ahat = A / ||A||_1``, k = 1..6) with ``||A||_1`` and ``||A||_inf``; the polynomial guess
``C_0 = ||A||_1^{-1/p} q(Ahat)`` for a cubic q, the degree-0 case being the scaled identity that Sec. 2
allows; its gate ``||I - C_0^p A||_2`` (Eq. 2) computed exactly by an eigensolver; the relative
least-squares cubic on a spectral interval that serves as a training label; and the 8-64-64-4 ReLU
network's forward pass, mean-squared loss and gradient written out layer by layer. Their pins
(tests/test_oracle_learned.py): traces from the known eigenvalues, C_0's eigenvalues equal q at the
eigenvalues, Eq. 3 and the scaled identity as special coefficient vectors, the gate against the scalar
model of Eq. 2, the fit on a vanishing interval, a hand-computed network case and central differences of
the loss.

Refinement (``refine_newton``, the section before the custom-precision functions): Newton's method on the
balanced residual ``I - sym(X^m A X^m')`` (m = floor(p/2), m' = p - m) with a conjugate-gradient solve of the
linearised equation, which corrects perturbations of any structure, the step Sec. 3 and Sec. 5 rely on to turn
an approximate result into a precise one. Its pins (tests/test_oracle_refine.py): on diagonal matrices every
entry follows the scalar Newton step for x^p a = 1; one correction equals the entry-wise solution in the
eigenbasis of a commuting X; a perturbed root converges quadratically to the closed form while the coupled
form started from it does not; planted mistakes in the linearised operator fail.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "norm_1", "norm_inf", "initial_guess_eq3", "initial_guess_scaled_identity", "symmetrize",
    "sym_product", "power_times", "residual_fro", "step_literal", "step_newton_schulz",
    "coupled_start", "step_coupled", "solve", "SolveInfo", "closed_form_root", "eig_root",
    "scalar_recurrence", "scalar_residuals", "forward_error", "default_form", "closed_form_block",
    "residual_rows", "eq2_prescale", "round_mantissa", "matmul_rounded", "quantized_iterates",
    "refine_operator", "refine_residual", "refine_correction", "refine_newton", "RefineInfo",
]


# ---------------------------------------------------------------- norms and initial guess (Eq. 3)

def norm_1(A: np.ndarray) -> float:
    """||A||_1: the largest absolute column sum, max_j sum_i |a_ij| (the 1-norm of Eq. 3)."""
    return float(np.max(np.sum(np.abs(A), axis=0)))


def norm_inf(A: np.ndarray) -> float:
    """||A||_inf: the largest absolute row sum, max_i sum_j |a_ij| (the infinity-norm of Eq. 3)."""
    return float(np.max(np.sum(np.abs(A), axis=1)))


def initial_guess_eq3(A: np.ndarray) -> np.ndarray:
    """Eq. 3: C_0 = (||A||_1 ||A||_inf)^{-1} A^T."""
    return np.ascontiguousarray(A.T / (norm_1(A) * norm_inf(A)))


def eq2_prescale(A: np.ndarray, p: int):
    """Reading of Eq. 2's scale caveat for Eq. 3's C_0 (the paper says Eq. 3 always satisfies Eq. 2).

    The eigenvalues of C_0^p A are lam^(p+1) / (||A||_1 ||A||_inf)^p <= ||A||_1^(1-p), so for p > 1 and
    ||A||_1 ||A||_inf < 1 Eq. 2 can fail (A = 0.1 I, p = 2: ||I - C_0^2 A||_2 = 9). Such an A is replaced by
    2^k A with ||2^k A||_1 = 2 f in [1, 2), where ||A||_1 = f 2^e, f in [0.5, 1), k = 1 - e; a power of two
    scales exactly, and A^{-1/p} = 2^(k/p) (2^k A)^{-1/p}. Returns (the matrix to iterate on, k); k = 0 leaves
    A as it is (p = 1, or ||A||_1 ||A||_inf >= 1).
    """
    if p <= 1 or norm_1(A) * norm_inf(A) >= 1.0:
        return A, 0
    _, e = np.frexp(norm_1(A))
    k = 1 - int(e)
    return np.ldexp(A, k), k


def initial_guess_scaled_identity(A: np.ndarray, p: int) -> np.ndarray:
    """The scalar start C_0 = ||A||_1^{-1/p} I, one of the "different possible choices" of Sec. 2.

    Because lambda_max(A) <= ||A||_1, the eigenvalues of C_0^p A lie in (0, 1], so Eq. 2 holds.
    """
    n = A.shape[0]
    return np.eye(n) * norm_1(A) ** (-1.0 / p)


# ---------------------------------------------------------------- products

def symmetrize(Y: np.ndarray) -> np.ndarray:
    """(Y + Y^T) / 2. The paper is silent on symmetrisation; every product here is symmetrised."""
    return 0.5 * (Y + Y.T)


def sym_product(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Product of two commuting symmetric matrices, symmetrised."""
    return symmetrize(X @ Y)


def power_times(C: np.ndarray, A: np.ndarray, p: int) -> np.ndarray:
    """C^p A, formed right to left: T = A, then p times T = C T (the order of Eq. 1's C_k^{p+1} A).

    No symmetrisation: for a C that does not commute with A exactly, C^j A is not symmetric.
    """
    T = A
    for _ in range(p):
        T = C @ T
    return T


def residual_fro(C: np.ndarray, A: np.ndarray, p: int) -> float:
    """||I - C^p A||_F, the Frobenius version of the quantity bounded in Eq. 2."""
    n = A.shape[0]
    return float(np.linalg.norm(np.eye(n) - power_times(C, A, p)))


# ---------------------------------------------------------------- one step of each form (Eq. 1)

def step_literal(C: np.ndarray, A: np.ndarray, p: int) -> np.ndarray:
    """Eq. 1 as printed: C' = ((p + 1) C - C^{p+1} A) / p, the result symmetrised."""
    T = power_times(C, A, p + 1)
    return symmetrize(((p + 1) * C - T) / p)


def step_newton_schulz(C: np.ndarray, A: np.ndarray) -> np.ndarray:
    """p = 1 (Sec. 2, Newton-Schulz): C' = 2C - C (A C), equal to Eq. 1 with p = 1 when C commutes with A.

    The inner product T = A C is kept unsymmetrised: its non-symmetric part is what makes the step
    correct errors that do not commute with A (C A C is symmetric for every symmetric C). Symmetrising T
    multiplies such errors by -(sqrt(rho) - 1/sqrt(rho))^2 / 4 per step, rho a ratio of eigenvalues of A.
    """
    T = A @ C
    return symmetrize(2.0 * C - C @ T)


def coupled_start(X0: np.ndarray, A: np.ndarray, p: int):
    """Coupled form: (X_0, M_0) with M_0 = X_0^p A; X_0 is a polynomial in A, so each product is symmetric."""
    M = A
    for _ in range(p):
        M = sym_product(X0, M)
    return X0.copy(), M


def step_coupled(X: np.ndarray, M: np.ndarray, p: int):
    """One coupled step: N = ((p+1) I - M) / p; X' = X N; M' = N^p M (p products, right to left)."""
    n = X.shape[0]
    N = ((p + 1) * np.eye(n) - M) / p
    Xn = sym_product(X, N)
    Mn = M
    for _ in range(p):
        Mn = sym_product(N, Mn)
    return Xn, Mn


# ---------------------------------------------------------------- the solve loop

def default_form(p: int) -> str:
    """Newton-Schulz for p = 1, the coupled order otherwise."""
    return "ns" if p == 1 else "coupled"


@dataclass
class SolveInfo:
    form: str
    c0: str
    p: int
    iterations: int = 0  # number of updates applied to C
    residuals: list = field(default_factory=list)  # r_0 .. r_k, r_k belongs to the returned iterate
    stop: str = ""  # "tol", "stagnation", "max_iter", "diverged" or (coupled form) "inaccurate"
    seconds: float = 0.0
    true_residual: float = -1.0  # ||I - C^p A||_F of the returned iterate (coupled form with verify)


def solve(A: np.ndarray, p: int, form: str | None = None, c0: str = "eq3", tol: float = 1e-12,
          max_iter: int = 100, stag_below: float = 1e-3, stag_ratio: float = 0.5,
          C0: np.ndarray | None = None, verify: bool = True):
    """Iterate Eq. 1 from C_0 until the residual meets ``tol``.

    Stop rule (reading; the paper gives none): after computing r_k for the current iterate, stop with
    "tol" if r_k <= tol; with "diverged" if r_k is not finite; with "stagnation" if r_{k-1} < stag_below
    and r_k > stag_ratio * r_{k-1}; with "max_iter" if k == max_iter. Otherwise apply one update.
    The returned iterate is the one whose residual was r_k.

    ``r_k`` is ||I - C_k^p A||_F for the literal and Newton-Schulz forms and ||I - M_k||_F for the
    coupled form (equal in exact arithmetic). With ``verify`` the coupled form then evaluates the true
    residual ||I - C^p A||_F of the returned iterate (reading: the residual Sec. 2 defines is the true one;
    rounding errors carried in M can separate the two), and a "tol" stop whose true residual exceeds
    ``tol`` becomes "inaccurate".
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    form = form or default_form(p)
    if form == "ns" and p != 1:
        raise ValueError("the Newton-Schulz form is the p = 1 case")
    if C0 is None:
        C0 = initial_guess_eq3(A) if c0 == "eq3" else initial_guess_scaled_identity(A, p)
        c0_name = c0
    else:
        c0_name = "given"
    info = SolveInfo(form=form, c0=c0_name, p=p)
    eye = np.eye(n)
    t0 = time.perf_counter()

    def decide(r: float, k: int) -> str:
        info.residuals.append(r)
        if not np.isfinite(r):
            return "diverged"
        if r <= tol:
            return "tol"
        if k >= 1 and info.residuals[-2] < stag_below and r > stag_ratio * info.residuals[-2]:
            return "stagnation"
        if k >= max_iter:
            return "max_iter"
        return ""

    C = np.array(C0, dtype=np.float64, copy=True)
    k = 0
    if form == "coupled":
        X, M = coupled_start(C, A, p)
        while True:
            stop = decide(float(np.linalg.norm(eye - M)), k)
            if stop:
                break
            X, M = step_coupled(X, M, p)
            k += 1
        C = X
    elif form == "ns":
        while True:
            T = A @ C
            stop = decide(float(np.linalg.norm(eye - T)), k)
            if stop:
                break
            C = symmetrize(2.0 * C - C @ T)
            k += 1
    elif form == "literal":
        while True:
            T = power_times(C, A, p)
            stop = decide(float(np.linalg.norm(eye - T)), k)
            if stop:
                break
            T = C @ T
            C = symmetrize(((p + 1) * C - T) / p)
            k += 1
    else:
        raise ValueError(f"unknown form {form!r}")
    info.iterations = k
    if form == "coupled" and verify and stop != "diverged":
        info.true_residual = residual_fro(C, A, p)
        if stop == "tol" and not info.true_residual <= tol:
            stop = "inaccurate"
    elif form != "coupled" and stop != "diverged":
        info.true_residual = info.residuals[-1]  # the Newton-Schulz and literal forms test the true residual
    info.stop = stop
    info.seconds = time.perf_counter() - t0
    return C, info


# ---------------------------------------------------------------- exact roots and the scalar recurrence

def closed_form_root(Q: np.ndarray, lam: np.ndarray, p: int) -> np.ndarray:
    """A^{-1/p} = Q diag(lam^{-1/p}) Q^T for A = Q diag(lam) Q^T (the limit named in Sec. 2)."""
    Z = (Q * lam ** (-1.0 / p)) @ Q.T
    return symmetrize(Z)


def closed_form_block(Q_rows: np.ndarray, Q_cols: np.ndarray, lam: np.ndarray, p: int) -> np.ndarray:
    """Entries Z[I, J] of Z = Q diag(lam^{-1/p}) Q^T from rows I and J of Q: the closed form of Sec. 2's limit
    evaluated one entry at a time, Z_ij = sum_k Q_ik lam_k^{-1/p} Q_jk (for orders too large to form Z)."""
    return (np.asarray(Q_rows) * lam ** (-1.0 / p)) @ np.asarray(Q_cols).T


def residual_rows(C: np.ndarray, A: np.ndarray, p: int, rows) -> np.ndarray:
    """Rows I of I - C^p A, formed as e_I^T - (((C[I] C) C) ... C) A with p - 1 factors C: the residual of
    Eq. 2 on a subset of rows, for orders where the full product is too large for the CPU."""
    rows = np.asarray(rows)
    T = np.array(C[rows], dtype=np.float64)
    for _ in range(p - 1):
        T = T @ C
    R = -(T @ A)
    R[np.arange(len(rows)), rows] += 1.0
    return R


def eig_root(A: np.ndarray, p: int) -> np.ndarray:
    """A^{-1/p} from a LAPACK symmetric eigendecomposition (a library routine, used as an independent pin)."""
    w, V = np.linalg.eigh(A)
    return symmetrize((V * w ** (-1.0 / p)) @ V.T)


def scalar_recurrence(lam: np.ndarray, c0: np.ndarray, p: int, k: int) -> np.ndarray:
    """Eigenvalues of C_k: Eq. 1 acts on each eigenvalue independently, c' = ((p + 1) c - c^{p+1} lam) / p."""
    c = np.array(c0, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    for _ in range(k):
        c = ((p + 1) * c - c ** (p + 1) * lam) / p
    return c


def scalar_residuals(lam: np.ndarray, c0: np.ndarray, p: int, k_max: int) -> np.ndarray:
    """||I - C_k^p A||_F = sqrt(sum_i (1 - c_k(lam_i)^p lam_i)^2) for k = 0..k_max (exact-arithmetic model)."""
    c = np.array(c0, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    out = []
    for _ in range(k_max + 1):
        out.append(float(np.sqrt(np.sum((1.0 - c ** p * lam) ** 2))))
        c = ((p + 1) * c - c ** (p + 1) * lam) / p
    return np.asarray(out)


def forward_error(C: np.ndarray, Z: np.ndarray) -> float:
    """||C - Z||_F / ||Z||_F, the Frobenius error of Sec. 4.3 made relative."""
    return float(np.linalg.norm(C - Z) / np.linalg.norm(Z))


# ---------------------------------------------------------------- refinement of an approximate root (Sec. 3, Sec. 5)
#
# Sec. 3 and Sec. 5: an approximation computed with imprecise arithmetic is refined into a precise root in a
# few additional precise iterations. For p = 1 Eq. 1's own step (Newton-Schulz) does that: it removes any
# perturbation of C to first order. For p >= 2 it does not: the coupled form keeps X_k M_k^{-1/p} fixed, so a
# perturbation that does not commute with A stays in the limit, amplified by up to about kappa / p.
# The refinement below is Newton's method on the balanced residual
#
#     G(X) = I - sym(X^m A X^m'),   m = floor(p / 2),  m' = p - m,
#
# whose solution near A^{-1/p} is A^{-1/p} (in the eigenbasis of a commuting X the residual is
# 1 - x^p lam). A step solves the linearised equation L_X(D) = G(X) for a symmetric correction D with
# L_X(D) = sym(dP_m(D) A X^m' + X^m A dP_m'(D)), where dP_k(D) = sum_{j<k} X^j D X^(k-1-j) is the first-order
# change of X^k, by conjugate gradients preconditioned with D = sym(X R) / p (the inverse of L_X on the
# diagonal of X's eigenbasis, where L_X multiplies by p x^(p-1) lam = p / x at the root), and sets
# X <- sym(X + D). Splitting X^p into two halves around A makes L_X a symmetric positive definite operator
# near the root with a spread of only about kappa^(1/2) between its eigenvalues (for p = 2 it is the Lyapunov
# operator D -> D A^(1/2) + A^(1/2) D).

def refine_operator(X: np.ndarray, A: np.ndarray, p: int, D: np.ndarray) -> np.ndarray:
    """L_X(D) = sym(dP_m(D) A X^m' + X^m A dP_m'(D)): the first-order change of sym(X^m A X^m') when X moves
    by D (m = floor(p / 2), m' = p - m, dP_k(D) = sum_{j<k} X^j D X^(k-1-j))."""
    m, mq = p // 2, p - p // 2

    def power(k):
        return np.linalg.matrix_power(X, k)

    def dpow(k):
        out = np.zeros_like(X)
        for j in range(k):
            out = out + power(j) @ D @ power(k - 1 - j)
        return out

    return symmetrize(dpow(m) @ A @ power(mq) + power(m) @ A @ dpow(mq))


def refine_residual(X: np.ndarray, A: np.ndarray, p: int) -> np.ndarray:
    """G(X) = I - sym(X^m A X^m'), m = floor(p / 2), m' = p - m."""
    m, mq = p // 2, p - p // 2
    F = np.linalg.matrix_power(X, m) @ A @ np.linalg.matrix_power(X, mq)
    return np.eye(A.shape[0]) - symmetrize(F)


def refine_correction(X: np.ndarray, A: np.ndarray, p: int, G: np.ndarray, cg_max: int = 50,
                      cg_tol: float = 1e-12):
    """The Newton correction: D with L_X(D) = G by conjugate gradients in the Frobenius inner product,
    preconditioned with R -> sym(X R) / p, from D = 0, until ||G - L_X(D)||_F <= cg_tol ||G||_F or cg_max
    iterations. Returns (D, iterations)."""
    def precondition(R):
        return symmetrize(X @ R) / p

    D = np.zeros_like(X)
    R = np.array(G, dtype=np.float64, copy=True)
    g0 = float(np.linalg.norm(G))
    if g0 == 0.0:
        return D, 0
    Zr = precondition(R)
    S = Zr.copy()
    rz = float(np.sum(R * Zr))
    it = 0
    while it < cg_max:
        LS = refine_operator(X, A, p, S)
        alpha = rz / float(np.sum(S * LS))
        D = D + alpha * S
        R = R - alpha * LS
        it += 1
        if float(np.linalg.norm(R)) <= cg_tol * g0:
            break
        Zr = precondition(R)
        rz_new = float(np.sum(R * Zr))
        S = Zr + (rz_new / rz) * S
        rz = rz_new
    return D, it


@dataclass
class RefineInfo:
    p: int
    steps: int = 0                                      # Newton corrections kept
    residuals: list = field(default_factory=list)       # ||G(X_k)||_F for k = 0 .. steps (last: returned X)
    cg_iterations: list = field(default_factory=list)   # CG iterations of each kept correction
    stop: str = ""        # "tol", "stagnation", "max_steps", "diverged" or "inaccurate"
    true_residual: float = -1.0                         # ||I - X^p A||_F of the returned X


def refine_newton(A: np.ndarray, X0: np.ndarray, p: int, max_steps: int = 8, tol: float = 1e-12,
                  cg_max: int = 50, cg_tol: float = 1e-12, stag_below: float = 1e-3, stag_ratio: float = 0.5):
    """Newton refinement of an approximate root X0 of A^{-1/p} (see the section comment).

    Before each step the residual g_k = ||G(X_k)||_F is recorded and tested: "tol" if g_k <= tol; if g_k is
    not finite or (k >= 1) g_k >= g_{k-1}, the last correction is undone (X and the record return to step
    k - 1) and the stop is "diverged" (not finite) or "stagnation"; "stagnation" also if g_{k-1} < stag_below
    and g_k > stag_ratio g_{k-1} (X_k kept); "max_steps" if k == max_steps. Otherwise one correction is
    applied. Afterwards the true residual ||I - X^p A||_F of the returned X is evaluated, and a "tol" stop
    whose true residual exceeds tol becomes "inaccurate". Returns (X, RefineInfo).
    """
    A = np.asarray(A, dtype=np.float64)
    X = symmetrize(np.asarray(X0, dtype=np.float64))
    info = RefineInfo(p=p)
    prev = None
    k = 0
    while True:
        G = refine_residual(X, A, p)
        g = float(np.linalg.norm(G))
        info.residuals.append(g)
        if not np.isfinite(g) or (k >= 1 and g >= info.residuals[-2]):
            stop = "diverged" if not np.isfinite(g) else "stagnation"
            if prev is not None:
                X = prev
                info.residuals.pop()
                info.cg_iterations.pop()
                k -= 1
            break
        if g <= tol:
            stop = "tol"
            break
        if k >= 1 and info.residuals[-2] < stag_below and g > stag_ratio * info.residuals[-2]:
            stop = "stagnation"
            break
        if k >= max_steps:
            stop = "max_steps"
            break
        D, its = refine_correction(X, A, p, G, cg_max, cg_tol)
        info.cg_iterations.append(its)
        prev = X
        X = symmetrize(X + D)
        k += 1
    info.steps = k
    if stop != "diverged":
        info.true_residual = residual_fro(X, A, p)
        if stop == "tol" and not info.true_residual <= tol:
            stop = "inaccurate"
    info.stop = stop
    return X, info


# ---------------------------------------------------------------- custom-precision simulation (Sec. 4.2, 4.3)
#
# The paper's experiment: the iteration with floating-point numbers of m stored mantissa bits, either for all
# involved calculations ("arithmetic") or only for the input and the stored intermediate results ("storage",
# approximate storage or data exchange), against the exact root (Fig. 2). Readings: the exponent range stays
# that of FP64 (only the mantissa is shortened); rounding is to nearest, ties to even; an operation in the
# custom type is the FP64 operation followed by that rounding; a product of matrices sums its terms in the
# order k = 0, 1, ..., n - 1, rounding every product and every partial sum; the iteration is Eq. 1 as printed
# (C^{p+1} A right to left, the new iterate symmetrised), from Eq. 3's C_0 computed in FP64 from the rounded
# input and then rounded; storage keeps A and each iterate rounded and computes in FP64.

def round_mantissa(x, m: int):
    """x rounded to m stored mantissa bits (m + 1 significant bits), ties to even: x = f 2^e with
    0.5 <= |f| < 1 becomes rint(f 2^(m+1)) 2^(e - m - 1)."""
    f, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(np.ldexp(f, m + 1)), e - m - 1)


def matmul_rounded(X: np.ndarray, Y: np.ndarray, m: int) -> np.ndarray:
    """X Y in the m-bit arithmetic: P_ij = (((x_i0 y_0j) + x_i1 y_1j) + ...), every product and every partial
    sum rounded to m bits."""
    P = np.zeros((X.shape[0], Y.shape[1]))
    for k in range(X.shape[1]):
        P = round_mantissa(P + round_mantissa(np.outer(X[:, k], Y[k, :]), m), m)
    return P


def quantized_iterates(A: np.ndarray, p: int, m: int, mode: str, iterations: int):
    """The literal iteration of Eq. 1 in the custom precision (mode "storage" or "arithmetic"); returns the
    iterates C_0 .. C_iterations. Arithmetic: every product term and sum (matmul_rounded), and the update
    ((p + 1) C - C^{p+1} A) / p and the symmetrisation (Y + Y^T) / 2 one rounded operation at a time."""
    rnd = lambda Y: round_mantissa(Y, m)  # noqa: E731
    Aq = rnd(A)
    C = rnd(initial_guess_eq3(Aq))
    out = [C]
    for _ in range(iterations):
        T = Aq
        for _ in range(p + 1):
            T = C @ T if mode == "storage" else matmul_rounded(C, T, m)
        if mode == "storage":
            C = rnd(symmetrize(((p + 1) * C - T) / p))
        else:
            W = rnd(rnd(rnd((p + 1) * C) - T) / p)
            C = rnd(W + W.T) * 0.5
        out.append(C)
    return out


# ---------------------------------------------------------------- learned polynomial initial guess
#
# A generalisation of the scalar start: C_0 = ||A||_1^{-1/p} q(A_hat), q(x) = c_0 + c_1 x + c_2 x^2 + c_3 x^3,
# A_hat = A / ||A||_1 (eigenvalues in (0, 1] for SPD A). Any such C_0 is a polynomial in A, so it commutes
# with A and the iterates of Eq. 1 remain polynomials in A; Eq. 2 must still hold, which a gate checks.

def spectral_features(A: np.ndarray) -> np.ndarray:
    """[tr(A_hat^k)/n for k = 1..6, ||A||_1, ||A||_inf], A_hat = A / ||A||_1 (definitions written out)."""
    n = A.shape[0]
    s = norm_1(A)
    Ah = A / s
    P = np.eye(n)
    out = []
    for _ in range(6):
        P = P @ Ah
        out.append(np.trace(P) / n)
    return np.array(out + [s, norm_inf(A)])


def polynomial_initial_guess(A: np.ndarray, p: int, c) -> np.ndarray:
    """C_0 = ||A||_1^{-1/p} (c_0 I + c_1 A_hat + c_2 A_hat^2 + c_3 A_hat^3)."""
    n = A.shape[0]
    s = norm_1(A)
    Ah = A / s
    P, C = np.eye(n), np.zeros((n, n))
    for ci in c:
        C = C + ci * P
        P = P @ Ah
    return symmetrize(C * s ** (-1.0 / p))


def gate_value(A: np.ndarray, p: int, C0: np.ndarray) -> float:
    """||I - C_0^p A||_2 (Eq. 2), from a LAPACK symmetric eigensolver of the symmetrised matrix."""
    E = np.eye(A.shape[0]) - np.linalg.matrix_power(C0, p) @ A
    return float(np.abs(np.linalg.eigvalsh(symmetrize(E))).max())


def relative_fit(lo: float, hi: float, p: int, degree: int = 3, points: int = 400) -> np.ndarray:
    """Coefficients c of q minimising sum_x (1 - q(x) x^{1/p})^2 over `points` log-spaced x in [lo, hi]:
    q(x)^p x close to 1 in the relative sense on the spectrum of A_hat, i.e. C_0^p A close to I."""
    x = np.exp(np.linspace(np.log(lo), np.log(hi), points))
    B = np.stack([x ** (i + 1.0 / p) for i in range(degree + 1)], axis=1)
    c, *_ = np.linalg.lstsq(B, np.ones(points), rcond=None)
    return c


# ---------------------------------------------------------------- the MLP (8 -> 64 -> 64 -> 4, ReLU), FP64
# Flat parameter layout (shared with the library): W1 (64 x 8), b1 (64), W2 (64 x 64), b2 (64), W3 (4 x 64), b3 (4).

MLP_SHAPES = [(64, 8), (64,), (64, 64), (64,), (4, 64), (4,)]
MLP_PARAMS = sum(int(np.prod(s)) for s in MLP_SHAPES)


def mlp_unpack(theta):
    out, k = [], 0
    for s in MLP_SHAPES:
        m = int(np.prod(s))
        out.append(np.asarray(theta[k:k + m], dtype=np.float64).reshape(s))
        k += m
    return out


def mlp_forward(theta, X):
    """Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for each row x of X."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(theta)
    H1 = np.maximum(X @ W1.T + b1, 0.0)
    H2 = np.maximum(H1 @ W2.T + b2, 0.0)
    return H2 @ W3.T + b3


def mlp_loss_grad(theta, X, T):
    """Mean squared error over all B x 4 outputs and its gradient (backpropagation written out)."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(theta)
    A1 = X @ W1.T + b1
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ W2.T + b2
    H2 = np.maximum(A2, 0.0)
    Y = H2 @ W3.T + b3
    B = X.shape[0]
    D = Y - T
    loss = float(np.sum(D * D) / (B * 4))
    dY = 2.0 * D / (B * 4)
    gW3, gb3 = dY.T @ H2, dY.sum(0)
    dA2 = (dY @ W3) * (A2 > 0)
    gW2, gb2 = dA2.T @ H1, dA2.sum(0)
    dA1 = (dA2 @ W2) * (A1 > 0)
    gW1, gb1 = dA1.T @ X, dA1.sum(0)
    return loss, np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])
