"""FP64-accurate products from exact FP16 digit slices (PR_EMU64), through the C ABI.

Product parity: each element is compared with the product evaluated in extended precision (numpy
longdouble). With S = 8 balanced base-256 digits per operand row (row exponent e_i: max_k |x_ik| <
2^(e_i - 1), digits |d| <= 128), the rounding of the rows to 8S bits contributes at most 2 2^(-8S - 2) and
the dropped digit pairs (s + t > S + 1) at most S 2^(-8S - 2) per product term, in units of 2^(e_i + f_j);
the level sums are exact and the total is rounded once to FP64, so over K = n terms the bound is
n (S + 2) 2^(-8S - 2) 2^(e_i + f_j) + 16 u |P_ij|,  u = 2^-53.
Solver parity: PR_EMU64 iterations meet the same bar as the native FP64 path against the CPU oracle.
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
S = 8
U = 2.0 ** -53


def row_exponents(X):
    m = np.abs(X).max(axis=1)
    _, p = np.frexp(m)  # m = f 2^p, 0.5 <= f < 1
    return np.where(m > 0, p + 1, 0)


def emu_bound(X, Y, ref, slices=S):
    n = X.shape[0]
    ex, ey = row_exponents(X), row_exponents(Y)
    scale = np.ldexp(1.0, ex[:, None] + ey[None, :])
    return n * (slices + 2) * 2.0 ** (-8 * slices - 2) * scale + 16 * U * np.abs(ref)


def sym_pair(n, seed):
    c = W.spd_from_spectrum(n, 0.05, seed)
    X = c.A / O.norm_1(c.A)
    Y = 0.5 * np.eye(n) + X @ X
    return np.ascontiguousarray(X), np.ascontiguousarray(0.5 * (Y + Y.T))


def gpu_matmul(prec, X, Y, sym):
    n = X.shape[0]
    Xd, Yd = torch.from_numpy(X).to(DEV), torch.from_numpy(Y).to(DEV)
    Pd = torch.empty_like(Xd)
    P.pr_matmul(prec, Xd, Yd, n, sym, Pd, torch.cuda.current_stream(DEV).cuda_stream)
    return Pd.cpu().numpy()


@pytest.mark.parametrize("n", [1, 8, 100, 128, 129, 257, 300])
@pytest.mark.parametrize("sym", [True, False])
def test_emu_product_elementwise(n, sym):
    X, Y = sym_pair(n, 60 + n)
    ref = (X.astype(np.longdouble) @ Y.T.astype(np.longdouble))  # K-major operands: X Y^T (= X Y)
    Pg = gpu_matmul(P.PR_EMU64, X, Y, sym)
    err = np.abs(Pg.astype(np.longdouble) - ref).astype(np.float64)
    bound = emu_bound(X, Y, ref.astype(np.float64))
    if sym:
        iu = np.triu_indices(n)
        assert np.all(err[iu] <= bound[iu])
        assert np.array_equal(Pg, Pg.T)
    else:
        assert np.all(err <= bound)


@pytest.mark.parametrize("slices", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("n,sym", [(129, True), (300, False)])
def test_emu_product_every_slice_count(slices, n, sym):
    # Every slice count the options allow: element-wise within the truncation bound of `slices` planes.
    X, Y = sym_pair(n, 90 + n)
    ref = (X.astype(np.longdouble) @ Y.T.astype(np.longdouble))
    Xd, Yd = torch.from_numpy(X).to(DEV), torch.from_numpy(Y).to(DEV)
    Pd = torch.empty_like(Xd)
    P.pr_matmul_emu(slices, Xd, Yd, n, sym, Pd, torch.cuda.current_stream(DEV).cuda_stream)
    Pg = Pd.cpu().numpy()
    err = np.abs(Pg.astype(np.longdouble) - ref).astype(np.float64)
    bound = emu_bound(X, Y, ref.astype(np.float64), slices)
    sel = np.triu_indices(n) if sym else np.indices((n, n)).reshape(2, -1)
    assert np.all(np.isfinite(Pg[sel]))
    assert np.all(err[sel] <= bound[sel]), (slices, float(np.max(err[sel] / bound[sel])))


@pytest.mark.parametrize("tile_n", [96, 48])
@pytest.mark.parametrize("split", [-1, 0, 1])
@pytest.mark.parametrize("n,sym", [(17, True), (129, True), (300, False), (700, True)])
def test_emu_product_every_variant(tile_n, split, n, sym):
    # Every work-list variant the tuner chooses between (tile width, whole or K-split tiles) gives the same
    # product: element-wise within the truncation bound, and bit-equal to the default variant.
    X, Y = sym_pair(n, 110 + n)
    ref = X.astype(np.longdouble) @ Y.T.astype(np.longdouble)
    Xd, Yd = torch.from_numpy(X).to(DEV), torch.from_numpy(Y).to(DEV)
    Pd = torch.empty_like(Xd)
    P.pr_matmul_emu_tiled(8, tile_n, split, Xd, Yd, n, sym, Pd, torch.cuda.current_stream(DEV).cuda_stream)
    Pg = Pd.cpu().numpy()
    err = np.abs(Pg.astype(np.longdouble) - ref).astype(np.float64)
    bound = emu_bound(X, Y, ref.astype(np.float64))
    sel = np.triu_indices(n) if sym else np.indices((n, n)).reshape(2, -1)
    assert np.all(err[sel] <= bound[sel])
    assert np.array_equal(Pg, gpu_matmul(P.PR_EMU64, X, Y, sym))


@pytest.mark.parametrize("tile", [0, 48])
def test_emu_solve_with_tuned_or_narrow_tiles(tile):
    # The tuner (tile 0) picks a variant per product kind; the narrow tiles can be fixed. Either way the solve
    # meets the oracle bar, and the stats report the width in use.
    case = W.spd_from_spectrum(300, 1e-2, 7)
    o = P.pr_default_options()
    o.emu_tile = tile
    A = torch.from_numpy(case.A).to(DEV)
    h = P.pr_init(A, 300, 2, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        P.pr_iterate(h, 100, P.PR_EMU64, 1e-12)
        C = torch.empty_like(A)
        P.pr_result(h, C)
        st = P.pr_stats(h)
    finally:
        P.pr_destroy(h)
    assert st["emu_tile_n"][0] in ((96, 48) if tile == 0 else (48,))
    Co, info = O.solve(case.A, 2, tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, 2)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C.cpu().numpy(), Z) <= bound


def test_emu_product_full_size_sampled():
    n = 4096
    c = W.spd_from_spectrum(n, 1e-3, 1)
    X = np.ascontiguousarray(c.A / O.norm_1(c.A))
    Pg = gpu_matmul(P.PR_EMU64, X, X, True)
    rng = np.random.default_rng(1)
    ii, jj = rng.integers(0, n, 1500), rng.integers(0, n, 1500)
    Xl = X.astype(np.longdouble)
    ref = np.einsum("ij,ij->i", Xl[ii], Xl[jj])
    ex = row_exponents(X)
    bound = n * (S + 2) * 2.0 ** (-8 * S - 2) * np.ldexp(1.0, ex[ii] + ex[jj]) + 16 * U * np.abs(ref.astype(np.float64))
    err = np.abs(Pg[ii, jj].astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err <= bound)
    assert np.array_equal(Pg, Pg.T)


def gpu_solve(case, p, prec, c0=P.PR_C0_EQ3, tol=1e-12, bulk=None, bulk_steps=0, slices=0):
    o = P.pr_default_options()
    o.c0 = c0
    o.emu_slices = slices
    A = torch.from_numpy(case.A).to(DEV)
    h = P.pr_init(A, case.n, p, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        st, steps = P.pr_solve(h, bulk if bulk is not None else prec, bulk_steps, prec, tol)
        C = torch.empty_like(A)
        P.pr_result(h, C)
        return C.cpu().numpy(), st, steps, P.pr_stats(h), P.pr_history(h)
    finally:
        P.pr_destroy(h)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_emu_solve_matches_oracle_small_case(p):
    case = W.spd_from_spectrum(256, 1e-2, 0)
    C, st, steps, stats, hist = gpu_solve(case, p, P.PR_EMU64)
    Co, info = O.solve(case.A, p, tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, p)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C, Co) <= bound and O.forward_error(C, Z) <= bound
    assert abs(steps - info.iterations) <= 1
    assert stats["iterations_by_precision"][P.PR_EMU64] == steps


@pytest.mark.parametrize("p", [1, 2, 3])
def test_emu_solve_seven_slices(p):
    # The 7-plane path on a well-conditioned case (kappa = 1e2), where the 56 bits kept per row still
    # cover the iterates' range within a row: the solve meets the same bar against the oracle. (At
    # kappa = 1e3, n = 4096 they do not: the default stays at 8 planes.)
    case = W.spd_from_spectrum(256, 1e-2, 0)
    C, st, steps, stats, hist = gpu_solve(case, p, P.PR_EMU64, slices=7)
    assert stats["emu_slices"] == 7 and st in (P.PR_OK, P.PR_ESTAGNATED, P.PR_EINACCURATE)
    Co, info = O.solve(case.A, p, tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, p)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C, Co) <= bound and O.forward_error(C, Z) <= bound
    assert abs(steps - info.iterations) <= 1


@pytest.mark.parametrize("n", [7, 65, 130, 300])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_emu_solve_ragged_scaled_identity(n, p):
    case = W.spd_from_spectrum(n, 0.02, 200 + n)
    C, st, steps, stats, hist = gpu_solve(case, p, P.PR_EMU64, c0=P.PR_C0_SCALED_I)
    Co, info = O.solve(case.A, p, c0="scaled_identity", tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, p)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C, Z) <= bound
    assert O.forward_error(C, Co) <= bound


@pytest.mark.parametrize("prec", [P.PR_FP64, P.PR_EMU64])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_scaled_identity_groupings_tight(prec, p):
    # From the scaled identity the oracle's own forward error is near 1e-14, so the bar max(1e-12, 10 x that)
    # is 1e-12: the two-product p = 3 update L R and the p = 4 grouping (N^2)^2 M are held to FP64 accuracy,
    # element by element on the whole result, and the stop is a verified PR_OK.
    case = W.spd_from_spectrum(256, 1e-2, 0)
    C, st, steps, stats, hist = gpu_solve(case, p, prec, c0=P.PR_C0_SCALED_I)
    Co, info = O.solve(case.A, p, c0="scaled_identity", tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, p)
    assert O.forward_error(Co, Z) < 1e-13
    bar = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C, Z) <= bar and O.forward_error(C, Co) <= bar
    assert np.max(np.abs(C - Co)) <= bar * np.max(np.abs(Co))
    assert abs(steps - info.iterations) <= 1
    assert st == {"tol": P.PR_OK, "stagnation": P.PR_ESTAGNATED, "inaccurate": P.PR_EINACCURATE}[info.stop]
    # Both true residuals sit at the rounding floor of an FP64 root (about 3e-13 here), which is mostly the
    # rounding of evaluating I - C^p A itself: EMU64 products round once per element and report less, so the
    # library's value is bounded by the oracle's (within a factor 3), not equal to it.
    assert 0 < stats["true_residual"] <= 3 * info.true_residual


def test_ns_ladder_bf16_then_emu64():
    # p = 1: BF16 bulk iterations, then FP64-accurate emulated ones, reach the FP64 oracle's accuracy.
    case = W.spd_from_spectrum(512, 1e-3, 14)
    C, st, steps, stats, hist = gpu_solve(case, 1, P.PR_EMU64, bulk=P.PR_BF16, bulk_steps=100)
    Co, info = O.solve(case.A, 1, tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, 1)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C, Z) <= bound
    assert stats["iterations_by_precision"][P.PR_BF16] > 0 and stats["iterations_by_precision"][P.PR_EMU64] > 0


def test_emu_true_residual():
    case = W.spd_from_spectrum(200, 0.02, 8)
    o = P.pr_default_options()
    A = torch.from_numpy(case.A).to(DEV)
    h = P.pr_init(A, 200, 2, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        P.pr_iterate(h, 100, P.PR_FP64, 1e-12)
        r64 = P.pr_residual(h, P.PR_FP64)
        remu = P.pr_residual(h, P.PR_EMU64)
        C = torch.empty_like(A)
        P.pr_result(h, C)
    finally:
        P.pr_destroy(h)
    want = O.residual_fro(C.cpu().numpy(), case.A, 2)
    assert abs(remu - want) <= 1e-2 * want + 1e-15
    assert abs(r64 - want) <= 1e-2 * want + 1e-15
