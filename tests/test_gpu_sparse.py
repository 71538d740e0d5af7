"""Block-sparse products with A (pr_options.block_sparse) on the sparse overlap stand-in of Sec. 4.1, through the
C ABI.

The overlap matrices of Sec. 4.1 get sparser as they grow (6.2 % non-zeros at N = 3072, 3.1 % at 6144). The
library restricts every tile of a digit-slice product with A to the K steps where the rows of A it reads are
non-zero. The steps it leaves out add exact zeros to exact digit sums, so every product, and so every solve, is
bit-identical to the dense one: the tests compare whole results, residual histories and features bit for bit,
and the roots of S^-1 (p = 1, Newton-Schulz) and S^-1/2 (p = 2, coupled form and refinement) against a LAPACK
root at the FP64 bar.
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
TOL = 1e-12


def run(S, p, block_sparse):
    n = S.shape[0]
    o = P.pr_default_options()
    o.block_sparse = block_sparse
    h = P.pr_init(torch.from_numpy(S).to(DEV), n, p, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        if p == 1:
            st, _ = P.pr_solve(h, P.PR_BF16, 100, P.PR_EMU64, TOL)
        else:
            P.pr_iterate(h, 100, P.PR_EMU64, TOL)
            st, _ = P.pr_refine(h, P.PR_EMU64, P.PR_BF16, 12, TOL, 40, 1e-2)
        res = P.pr_residual(h, P.PR_EMU64)
        C = torch.empty((n, n), dtype=torch.float64, device=DEV)
        P.pr_result(h, C)
        out = dict(C=C.cpu().numpy(), status=st, residual=res, history=P.pr_history(h), stats=P.pr_stats(h),
                   features=P.pr_features(h))
    finally:
        P.pr_destroy(h)
    return out


def check_pair(S, p):
    sp, de = run(S, p, 1), run(S, p, 0)
    assert sp["stats"]["sparse_keep"] < 0.875 and sp["stats"]["sparse_products"] > 0
    assert de["stats"]["sparse_keep"] == 1.0 and de["stats"]["sparse_products"] == 0
    assert np.array_equal(sp["C"], de["C"])
    assert sp["history"] == de["history"] and sp["residual"] == de["residual"]
    assert sp["features"] == de["features"] and sp["status"] == de["status"]
    if p >= 2:
        assert sp["stats"]["refine_residuals"] == de["stats"]["refine_residuals"]
    return sp


@pytest.mark.parametrize("n,density", [(600, 0.15), (1536, W.PAPER_OVERLAP_DENSITY[1536])])
@pytest.mark.parametrize("p", [1, 2])
def test_block_sparse_solves_are_bit_identical(n, density, p):
    S, _ = W.sparse_overlap(n, density, 11 + n)
    sp = check_pair(S, p)
    assert O.forward_error(sp["C"], O.eig_root(S, p)) <= 1e-12


def test_dense_matrices_run_dense_products():
    c = W.spd_from_spectrum(300, 1e-2, 4)
    out = run(c.A, 2, 1)
    assert out["stats"]["sparse_keep"] == 1.0 and out["stats"]["sparse_products"] == 0


def test_zero_rows_blocks_and_tiny_orders():
    # A block-diagonal SPD matrix: off-diagonal tiles whose rows of A are zero in a whole block of K steps, and
    # orders below one tile.
    for n in (40, 300):
        c = W.spd_from_spectrum(n // 2, 1e-1, n)
        A = np.zeros((n, n))
        A[: n // 2, : n // 2] = c.A
        A[n // 2:, n // 2:] = 2.0 * c.A
        A = np.ascontiguousarray(A)
        for p in (1, 2):
            sp, de = run(A, p, 1), run(A, p, 0)
            assert np.array_equal(sp["C"], de["C"]) and sp["history"] == de["history"]
            assert O.forward_error(sp["C"], O.eig_root(A, p)) <= 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_paper_density_n3072(p):
    S, _ = W.sparse_overlap(3072, W.PAPER_OVERLAP_DENSITY[3072], 3072)
    sp = check_pair(S, p)
    assert sp["stats"]["sparse_keep"] < 0.6
    assert O.forward_error(sp["C"], O.eig_root(S, p)) <= 1e-12
