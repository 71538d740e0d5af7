"""The BF16 tcgen05 product kernel and the low-precision iterations, through the C ABI.

Kernel parity: P = X Y computed from BF16-rounded X and Y with FP32 accumulation is compared element by
element with the exact (FP64) product of the same BF16 values. Every BF16 x BF16 product is exact in FP32,
so the only error is the FP32 accumulation over K = n terms, bounded by gamma_n * (|X_b| |Y_b|)_ij with
gamma_n = n u / (1 - n u), u = 2^-24 (Higham, Accuracy and Stability, Thm 3.5); the test uses that bound.
"""
import numpy as np
import pytest

from oracle import pthroot_oracle as O
from paper_1703_02283_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1703_02283_gb300 import pthroot as P  # noqa: E402

DEV = torch.device("cuda:0")
U32 = 2.0 ** -24


def bf16(x: np.ndarray) -> np.ndarray:
    """Round each double to the nearest value with 8 significant bits (ties to even), returned as FP64.

    Written from the definition (x = m 2^e with 0.5 <= |m| < 1, keep rint(m 2^8) / 2^8) so that it rounds
    once; converting through FP32 first (as a float64 -> bfloat16 cast may) rounds twice and can differ.
    BF16 range limits do not matter for the values used here.
    """
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def gamma(n):
    return n * U32 / (1 - n * U32)


def sym_pair(n, seed):
    """Two commuting symmetric matrices (polynomials in one SPD matrix)."""
    c = W.spd_from_spectrum(n, 0.05, seed)
    X = c.A / O.norm_1(c.A)
    Y = 0.5 * np.eye(n) + X @ X
    Y = 0.5 * (Y + Y.T)
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def gpu_matmul(prec, X, Y, sym):
    n = X.shape[0]
    Xd, Yd = torch.from_numpy(X).to(DEV), torch.from_numpy(Y).to(DEV)
    Pd = torch.empty_like(Xd)
    P.pr_matmul(prec, Xd, Yd, n, sym, Pd, torch.cuda.current_stream(DEV).cuda_stream)
    return Pd.cpu().numpy()


@pytest.mark.parametrize("n", [1, 8, 100, 128, 129, 255, 256, 300, 520])
@pytest.mark.parametrize("sym", [True, False])
def test_bf16_product_elementwise(n, sym):
    X, Y = sym_pair(n, 40 + n)
    Xb, Yb = bf16(X), bf16(Y)
    ref = Xb @ Yb.T  # the kernel computes X Y^T (= X Y here) from K-major operands
    bound = gamma(n) * (np.abs(Xb) @ np.abs(Yb).T) + 1e-300
    Pg = gpu_matmul(P.PR_BF16, X, Y, sym)
    if sym:
        # upper triangle computed, lower mirrored: compare the upper triangle, then exact symmetry
        iu = np.triu_indices(n)
        assert np.all(np.abs(Pg[iu] - ref[iu]) <= bound[iu])
        assert np.array_equal(Pg, Pg.T)
    else:
        assert np.all(np.abs(Pg - ref) <= bound)


@pytest.mark.parametrize("n", [64, 200, 256])
def test_fp64_product_elementwise(n):
    X, Y = sym_pair(n, 7 + n)
    ref = X @ Y
    bound = 2 * n * 1.2e-16 * (np.abs(X) @ np.abs(Y))
    for sym in (True, False):
        Pg = gpu_matmul(P.PR_FP64, X, Y, sym)
        iu = np.triu_indices(n)
        assert np.all(np.abs(Pg[iu] - ref[iu]) <= bound[iu])
        if sym:
            assert np.array_equal(Pg, Pg.T)


def test_bf16_product_full_size_sampled():
    # The n = 4096 product in the symmetric launch configuration the solver uses; 4000 sampled outputs
    # checked one by one against the exact dot products of the BF16-rounded rows.
    n = 4096
    c = W.spd_from_spectrum(n, 1e-3, 1)
    X = np.ascontiguousarray(c.A / O.norm_1(c.A))
    Xb = bf16(X)
    Pg = gpu_matmul(P.PR_BF16, X, X, True)
    rng = np.random.default_rng(0)
    ii, jj = rng.integers(0, n, 4000), rng.integers(0, n, 4000)
    ref = np.einsum("ij,ij->i", Xb[ii], Xb[jj])
    bound = gamma(n) * np.einsum("ij,ij->i", np.abs(Xb[ii]), np.abs(Xb[jj]))
    assert np.all(np.abs(Pg[ii, jj] - ref) <= bound)
    assert np.array_equal(Pg, Pg.T)


def _solve(case, p, bulk, bulk_steps, final, tol=1e-12, c0=P.PR_C0_EQ3):
    o = P.pr_default_options()
    o.c0 = c0
    A = torch.from_numpy(case.A).to(DEV)
    h = P.pr_init(A, case.n, p, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        st, steps = P.pr_solve(h, bulk, bulk_steps, final, tol)
        C = torch.empty_like(A)
        P.pr_result(h, C)
        return C.cpu().numpy(), st, steps, P.pr_stats(h), P.pr_history(h)
    finally:
        P.pr_destroy(h)


def test_ns_ladder_bf16_then_fp64_matches_oracle():
    # p = 1 (Newton-Schulz) corrects errors of any kind, so BF16 bulk iterations followed by FP64 ones
    # reach the FP64 oracle's accuracy (the refinement claim of Sec. 3 and Sec. 5).
    case = W.spd_from_spectrum(256, 1e-2, 0)
    C, st, steps, stats, hist = _solve(case, 1, P.PR_BF16, 100, P.PR_FP64)
    Co, info = O.solve(case.A, 1, tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, 1)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C, Z) <= bound
    assert O.forward_error(C, Co) <= bound
    assert stats["iterations_by_precision"][P.PR_BF16] > 0 and stats["iterations_by_precision"][P.PR_FP64] > 0
    assert stats["switch_iteration"] == stats["iterations_by_precision"][P.PR_BF16]


@pytest.mark.parametrize("p", [1, 2, 3])
def test_bf16_only_approximate_end(p):
    # Pure BF16 iterations stop on their floor (stagnation); the result is an approximate root whose
    # error is stated against the exact root: below 10 * u_bf16 * kappa (u_bf16 = 2^-8).
    case = W.spd_from_spectrum(256, 0.1, 12)
    C, st, steps, stats, hist = _solve(case, p, P.PR_BF16, 0, P.PR_BF16, tol=1e-12, c0=P.PR_C0_SCALED_I)
    Z = O.closed_form_root(case.Q, case.lam, p)
    assert st in (P.PR_ESTAGNATED, P.PR_OK)
    assert O.forward_error(C, Z) <= 10 * 2.0 ** -8 * case.kappa
    assert np.array_equal(C, C.T)


def test_bf16_residual_history_follows_oracle_early():
    # While the residual is far above the BF16 floor the low-precision iteration tracks the FP64 one.
    case = W.spd_from_spectrum(300, 0.05, 13)
    C, st, steps, stats, hist = _solve(case, 2, P.PR_BF16, 0, P.PR_BF16, tol=1e-12, c0=P.PR_C0_SCALED_I)
    Co, info = O.solve(case.A, 2, c0="scaled_identity", tol=1e-12)
    ho = np.asarray(info.residuals)
    for k in range(min(4, len(hist), len(ho))):
        assert abs(hist[k] - ho[k]) <= 0.05 * ho[k] + 1e-2
