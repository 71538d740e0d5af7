"""The FP8 (E4M3) tcgen05 product, the split-FP32 product (PR_FP32X) and the precision ladder built on them,
through the C ABI.

FP8 product parity. Each row of X (and of Y, the B operand) is scaled by a power of two 2^-s_i with s_i the
exponent of the row's largest magnitude minus 7 (so that it maps into [128, 256)), rounded to E4M3 (3
mantissa bits, subnormals down to 2^-9, largest finite 448) to nearest even, multiplied on the tensor cores
with FP32 accumulation and scaled back by 2^(s_i + s_j). The reference is written here from that definition:
the rounding from frexp / rint (one rounding from FP64), the scales from frexp of the row maxima. Every
E4M3 x E4M3 product is exact in FP32 and the scaling by powers of two is exact, so the only error is the
FP32 accumulation over K = n terms: at most gamma_n (|Xq| |Yq|^T)_ij, gamma_n = n u / (1 - n u), u = 2^-24
(Higham, Accuracy and Stability, Thm 3.5). With Y = I every output is a single exact term: the product is
the quantised X itself, bit for bit, which checks the rounding (ties, subnormals) element by element.

PR_FP32X parity: the first 3 of the 8 balanced base-256 digit planes of each row. Dropping planes 4..8 moves
an element by at most 128 (256^-4 + 256^-5 + ...) < 1.004 x 2^-25 in units of its row scale, against
2^-25 for a rounding to 3 digits, so the PR_EMU64 truncation bound with S = 3, widened by 1 %, holds.
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
U53 = 2.0 ** -53


def e4m3(x):
    """Nearest E4M3 value (ties to even) of each double, saturating at 448, as FP64: |x| = m 2^e with
    0.5 <= m < 1 lies in the binade [2^(e-1), 2^e), whose E4M3 spacing is 2^(max(e - 1, -6) - 3)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)
    step = np.maximum(e - 1, -6) - 3
    r = np.ldexp(np.rint(np.ldexp(a, -step)), step)
    r = np.where(a == 0, 0.0, np.minimum(r, 448.0))
    return np.copysign(r, x)


def row_scales(X):
    """s_i = (exponent of max_k |x_ik|) - 7 with exponent = floor(log2(.)); 0 for a zero row."""
    m = np.abs(X).max(axis=1)
    _, e = np.frexp(m)
    return np.where(m > 0, (e - 1) - 7, 0)


def quantise(X):
    s = row_scales(X)
    return np.ldexp(e4m3(np.ldexp(X, -s[:, None])), s[:, None])


def gamma(n):
    return n * U32 / (1 - n * U32)


def sym_pair(n, seed):
    c = W.spd_from_spectrum(n, 0.05, seed)
    X = c.A / O.norm_1(c.A)
    Y = 0.5 * np.eye(n) + X @ X
    return np.ascontiguousarray(X), np.ascontiguousarray(0.5 * (Y + Y.T))


def gpu_matmul(prec, X, Y, sym):
    n = X.shape[0]
    Xd, Yd = torch.from_numpy(np.ascontiguousarray(X)).to(DEV), torch.from_numpy(np.ascontiguousarray(Y)).to(DEV)
    Pd = torch.empty_like(Xd)
    P.pr_matmul(prec, Xd, Yd, n, sym, Pd, torch.cuda.current_stream(DEV).cuda_stream)
    return Pd.cpu().numpy()


def test_e4m3_reference_on_known_values():
    # The test's own rounding against hand-checked E4M3 values (spacing 1/8 in [1, 2), 2^-9 below 2^-6).
    x = np.array([1.0625, 1.1875, 1.124, 200.0, 3 * 2.0 ** -9, 2.5 * 2.0 ** -9, 3.5 * 2.0 ** -9, 2.0 ** -11,
                  0.75 * 2.0 ** -9, 460.0, -1.0625, 15.5 * 2.0 ** -4, 2.0 ** -6 * 1.0625])
    want = np.array([1.0, 1.25, 1.125, 192.0, 3 * 2.0 ** -9, 2 * 2.0 ** -9, 4 * 2.0 ** -9, 0.0, 2.0 ** -9, 448.0,
                     -1.0, 1.0, 2.0 ** -6])
    np.testing.assert_array_equal(e4m3(x), want)


def test_fp8_quantiser_exact_through_identity():
    # X I^T = X quantised: one exact term per output. Rows hold ties at every spacing, subnormal-range
    # values relative to the row maximum, zeros and a zero row.
    rng = np.random.default_rng(5)
    n = 200
    X = rng.standard_normal((n, n)) * np.exp(rng.uniform(-12, 4, (n, 1)))
    for i in range(0, n, 7):  # exact ties of the row's E4M3 grid
        top = np.abs(X[i]).max()
        _, e = np.frexp(top)
        s = (e - 1) - 7
        X[i, 1:9] = np.ldexp(np.array([1.0625, 1.1875, 1.3125, 2.5 * 2.0 ** -9 * 64, 3.5 * 2.0 ** -3,
                                       2.5 * 2.0 ** -9, 0.75 * 2.0 ** -9, 2.0 ** -12]), s)
    X[3] = 0.0
    X[:, 17] = 0.0
    Pg = gpu_matmul(P.PR_FP8, X, np.eye(n), False)
    np.testing.assert_array_equal(Pg, quantise(X))


@pytest.mark.parametrize("n", [1, 8, 100, 128, 129, 255, 256, 300, 520])
@pytest.mark.parametrize("sym", [True, False])
def test_fp8_product_elementwise(n, sym):
    X, Y = sym_pair(n, 140 + n)
    Xq, Yq = quantise(X), quantise(Y)
    ref = Xq @ Yq.T
    bound = gamma(n) * (np.abs(Xq) @ np.abs(Yq).T) + 1e-300
    Pg = gpu_matmul(P.PR_FP8, X, Y, sym)
    sel = np.triu_indices(n) if sym else np.indices((n, n)).reshape(2, -1)
    err = np.abs(Pg[sel] - ref[sel])
    assert np.all(err <= bound[sel]), float(np.max(err / bound[sel]))
    if sym:
        assert np.array_equal(Pg, Pg.T)


def test_fp8_product_full_size_sampled():
    # The n = 4096 symmetric product of the single-matrix workload; 4000 sampled outputs one by one.
    n = 4096
    c = W.spd_from_spectrum(n, 1e-3, 1)
    X = np.ascontiguousarray(c.A / O.norm_1(c.A))
    Xq = quantise(X)
    Pg = gpu_matmul(P.PR_FP8, X, X, True)
    rng = np.random.default_rng(3)
    ii, jj = rng.integers(0, n, 4000), rng.integers(0, n, 4000)
    ref = np.einsum("ij,ij->i", Xq[ii], Xq[jj])
    bound = gamma(n) * np.einsum("ij,ij->i", np.abs(Xq[ii]), np.abs(Xq[jj]))
    assert np.all(np.abs(Pg[ii, jj] - ref) <= bound)


def fp32x_bound(X, Y, ref):
    n = X.shape[0]
    m = np.abs(X).max(axis=1)
    _, px = np.frexp(m)
    ex = np.where(m > 0, px + 1, 0)
    m = np.abs(Y).max(axis=1)
    _, py = np.frexp(m)
    ey = np.where(m > 0, py + 1, 0)
    scale = np.ldexp(1.0, ex[:, None] + ey[None, :])
    return 1.01 * n * 5 * 2.0 ** (-8 * 3 - 2) * scale + 16 * U53 * np.abs(ref)


@pytest.mark.parametrize("n,sym", [(1, True), (129, True), (300, False), (520, True)])
def test_fp32x_product_elementwise(n, sym):
    X, Y = sym_pair(n, 170 + n)
    ref = X.astype(np.longdouble) @ Y.T.astype(np.longdouble)
    Pg = gpu_matmul(P.PR_FP32X, X, Y, sym)
    err = np.abs(Pg.astype(np.longdouble) - ref).astype(np.float64)
    bound = fp32x_bound(X, Y, ref.astype(np.float64))
    sel = np.triu_indices(n) if sym else np.indices((n, n)).reshape(2, -1)
    assert np.all(err[sel] <= bound[sel]), float(np.max(err[sel] / bound[sel]))


def solve(case, p, precisions, max_steps=None, c0=P.PR_C0_EQ3, tol=1e-12):
    o = P.pr_default_options()
    o.c0 = c0
    A = torch.from_numpy(case.A).to(DEV)
    h = P.pr_init(A, case.n, p, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        st, steps = P.pr_solve_ladder(h, precisions, max_steps, tol)
        C = torch.empty_like(A)
        P.pr_result(h, C)
        return C.cpu().numpy(), st, steps, P.pr_stats(h), P.pr_history(h)
    finally:
        P.pr_destroy(h)


def test_ns_ladder_fp8_bf16_emu64():
    # p = 1 (Newton-Schulz corrects earlier errors to first order): FP8 bulk, then BF16, then FP64-accurate
    # EMU64 iterations reach the FP64 oracle's accuracy; every rung ran.
    case = W.spd_from_spectrum(512, 1e-3, 14)
    C, st, steps, stats, hist = solve(case, 1, [P.PR_FP8, P.PR_BF16, P.PR_EMU64])
    Co, info = O.solve(case.A, 1, tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, 1)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C, Z) <= bound
    by = stats["iterations_by_precision"]
    assert by[P.PR_FP8] > 0 and by[P.PR_EMU64] > 0, by
    assert steps == sum(by)


def test_fp8_residual_tracks_oracle_early():
    # While the residual is far above the FP8 floor the FP8 iteration follows the FP64 one.
    case = W.spd_from_spectrum(300, 0.05, 13)
    C, st, steps, stats, hist = solve(case, 1, [P.PR_FP8], c0=P.PR_C0_EQ3)
    Co, info = O.solve(case.A, 1, tol=1e-12)
    ho = np.asarray(info.residuals)
    for k in range(min(3, len(hist))):
        assert abs(hist[k] - ho[k]) <= 0.15 * ho[k] + 0.1, (k, hist[k], ho[k])
    assert st == P.PR_ESTAGNATED


@pytest.mark.parametrize("p", [1, 2, 3])
def test_fp32x_only_approximate_end(p):
    # Pure PR_FP32X iterations from the scaled identity stop on their floor (the low-precision stop rule);
    # the result is an approximate root. Stated bound: a product's error per element is up to 2^-25 per
    # term relative to the row and column scales, about sqrt(n) 2^-25 over n terms of mixed signs, and the
    # iteration's attainable accuracy is that times kappa: forward error <= 10 sqrt(n) 2^-25 kappa. For p = 1
    # EMU64 iterations after them refine to the FP64 bar (Newton-Schulz corrects earlier errors).
    case = W.spd_from_spectrum(256, 1e-2, 15)
    Z = O.closed_form_root(case.Q, case.lam, p)
    C, st, steps, stats, hist = solve(case, p, [P.PR_FP32X], c0=P.PR_C0_SCALED_I)
    assert st in (P.PR_ESTAGNATED, P.PR_OK, P.PR_EINACCURATE)
    fe = O.forward_error(C, Z)
    assert fe <= 10 * np.sqrt(case.n) * 2.0 ** -25 * case.kappa, fe
    assert stats["iterations_by_precision"][P.PR_FP32X] == steps
    if p == 1:
        C2, st2, _, stats2, _ = solve(case, 1, [P.PR_FP32X, P.PR_EMU64], c0=P.PR_C0_SCALED_I)
        Co, info = O.solve(case.A, 1, c0="scaled_identity", tol=1e-12)
        assert O.forward_error(C2, Z) <= max(1e-12, 10 * O.forward_error(Co, Z))


def test_large_recipe_ladder_reports_its_error():
    # The ladder of the large recipe (FP8 bulk, then BF16, then split-FP32) on an order-1024 instance
    # (kappa = 1e4, p = 2, scaled identity start). For p >= 2 an early low-precision error is carried, not
    # refined away (the coupled form's final iterate is X M^{-1/p}); the result is an approximate end whose
    # error is measured and reported, not a FP64-accurate root. The test checks that no rung diverges (a
    # low-precision rung stops and rolls back at its first residual increase), that the counts of every rung
    # add up, and that the result is an approximation at all (relative error below 1).
    case = W.spd_from_spectrum(1024, 1e-4, 22)
    Z = O.closed_form_root(case.Q, case.lam, 2)
    C, st, steps, stats, hist = solve(case, 2, [P.PR_FP8, P.PR_BF16, P.PR_FP32X], c0=P.PR_C0_SCALED_I)
    by = stats["iterations_by_precision"]
    assert st != P.PR_EDIVERGED and np.all(np.isfinite(C))
    assert steps == by[P.PR_FP8] + by[P.PR_BF16] + by[P.PR_FP32X]
    fe = O.forward_error(C, Z)
    print("large-recipe ladder at n = 1024:", by, P.STATUS_NAMES[st], "forward error", fe)
    assert fe < 1.0


@pytest.mark.parametrize("n, seed", [(1024, 22), (2048, 23)])
def test_ladder_guard_keeps_the_best_iterate(n, seed):
    # The rung guard of pr_solve_ladder: after the ladder of the large recipe (FP8, BF16, split-FP32) from the
    # scaled identity at kappa = 1e4, p = 2, the true residual of the result (FP64-accurate products) is no
    # larger than the starting iterate's, whatever the carried ||I - M||_F of a low-precision rung said; the
    # counts of every rung still add up.
    case = W.spd_from_spectrum(n, 1e-4, seed)
    A = torch.from_numpy(case.A).to(DEV)
    o = P.pr_default_options()
    o.c0 = P.PR_C0_SCALED_I
    h = P.pr_init(A, n, 2, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        r0 = P.pr_residual(h, P.PR_EMU64)
        st, steps = P.pr_solve_ladder(h, [P.PR_FP8, P.PR_BF16, P.PR_FP32X], None, 1e-12)
        stats = P.pr_stats(h)
        r1 = P.pr_residual(h, P.PR_EMU64)
    finally:
        P.pr_destroy(h)
    by = stats["iterations_by_precision"]
    print(f"n = {n}: start {r0:.3e}, ladder end {r1:.3e}, restores {stats['ladder_restores']}, {by}")
    assert st != P.PR_EDIVERGED
    assert np.isfinite(r1) and r1 <= r0 * (1 + 1e-3)
    assert 0 <= stats["ladder_restores"] <= 3
    assert steps == by[P.PR_FP8] + by[P.PR_BF16] + by[P.PR_FP32X]


def test_ladder_ending_in_emu64_reaches_fp64_accuracy():
    # The large recipe's ladder with an FP64-accurate last rung (kappa = 1e4, p = 2, order 1024, scaled
    # identity start): whatever the low-precision rungs leave, the last rung ends at the FP64 oracle's
    # accuracy (a rung that diverges from their iterate restarts from the starting one).
    case = W.spd_from_spectrum(1024, 1e-4, 22)
    Z = O.closed_form_root(case.Q, case.lam, 2)
    C, st, steps, stats, hist = solve(case, 2, [P.PR_FP8, P.PR_BF16, P.PR_FP32X, P.PR_EMU64],
                                      c0=P.PR_C0_SCALED_I)
    Co, info = O.solve(case.A, 2, tol=1e-12, c0="scaled_identity")
    by = stats["iterations_by_precision"]
    fe, feo = O.forward_error(C, Z), O.forward_error(Co, Z)
    print("ladder ending in EMU64:", by, P.STATUS_NAMES[st], "restores", stats["ladder_restores"], "forward error",
          fe, "oracle", feo)
    assert st in (P.PR_OK, P.PR_ESTAGNATED, P.PR_EINACCURATE)
    assert by[P.PR_EMU64] > 0 and steps == sum(by)
    assert fe <= max(1e-12, 10 * feo)
