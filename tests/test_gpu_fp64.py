"""Parity of the native FP64 GPU path with the CPU oracle, through the C ABI.

Bar: the GPU iterate's relative Frobenius distance to the oracle's iterate, and to the exact root, is at
most max(1e-12, 10 x the oracle's own forward error); the iteration counts agree within one step; the
residual histories agree (rtol 1e-8) while they are well above the FP64 floor.
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
FORMS = {"auto": P.PR_FORM_AUTO, "coupled": P.PR_FORM_COUPLED, "ns": P.PR_FORM_NS, "literal": P.PR_FORM_LITERAL}
C0S = {"eq3": P.PR_C0_EQ3, "scaled_identity": P.PR_C0_SCALED_I}


def gpu_solve(A_np, p, form="auto", c0="eq3", tol=1e-12, max_iter=100, precision=P.PR_FP64, host=False,
              stag_below=1e-3):
    n = A_np.shape[0]
    o = P.pr_default_options()
    o.form = FORMS[form]
    o.c0 = C0S[c0]
    o.max_iter = max_iter
    o.stag_below = stag_below
    stream = torch.cuda.current_stream(DEV).cuda_stream
    if host:
        A = np.ascontiguousarray(A_np)
        h = P.pr_init(A, n, p, o, stream)
    else:
        A = torch.from_numpy(A_np).to(DEV)
        h = P.pr_init(A, n, p, o, stream)
    try:
        st, steps = P.pr_iterate(h, max_iter, precision, tol)
        if host:
            C = np.empty((n, n))
            P.pr_result(h, C)
        else:
            Ct = torch.empty((n, n), dtype=torch.float64, device=DEV)
            P.pr_result(h, Ct)
            C = Ct.cpu().numpy()
        return C, st, steps, P.pr_history(h), P.pr_stats(h), h
    except Exception:
        P.pr_destroy(h)
        raise


def check_parity(case, p, form="auto", c0="eq3", tol=1e-12, **kw):
    Co, info = O.solve(case.A, p, form=None if form == "auto" else form, c0=c0, tol=tol)
    C, st, steps, hist, stats, h = gpu_solve(case.A, p, form, c0, tol, **kw)
    P.pr_destroy(h)
    Z = O.closed_form_root(case.Q, case.lam, p)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert np.array_equal(C, C.T)
    assert O.forward_error(C, Co) <= bound, (O.forward_error(C, Co), bound)
    assert O.forward_error(C, Z) <= bound
    assert abs(steps - info.iterations) <= 1, (steps, info.iterations, info.stop)
    floor = O.residual_fro(Z, case.A, p)
    ho, hg = np.asarray(info.residuals), np.asarray(hist)
    m = min(len(ho), len(hg))
    mask = ho[:m] > 1e3 * floor
    # Two FP64 runs of the iteration differ by roundoff amplified by the spread of M_0 = C_0^p A: its
    # eigenvalues lam^{p+1}/s^p span kappa^{p+1} from Eq. 3's guess and kappa from the scaled identity.
    # The residual evaluations themselves differ by roundoff of the order of the FP64 floor.
    kappa = case.lam.max() / case.lam.min()
    spread = kappa ** (p + 1) if c0 == "eq3" else kappa
    rtol = max(1e-8, 10 * 2.2e-16 * spread)
    np.testing.assert_allclose(hg[:m][mask], ho[:m][mask], rtol=rtol, atol=10 * floor)
    return C, Co, steps, stats


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_small_case_recipe(p):
    # n = 256, kappa = 1e2 (the recipe the oracle finishes in seconds), Eq. 3 start.
    case = W.spd_from_spectrum(256, 1e-2, 0)
    check_parity(case, p)


@pytest.mark.parametrize("n", [1, 7, 63, 64, 65, 130, 200])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_ragged_sizes(n, p):
    case = W.spd_from_spectrum(n, 0.05, 100 + n)
    check_parity(case, p, c0="scaled_identity")


@pytest.mark.parametrize("p", [1, 2, 3])
def test_literal_form_well_conditioned(p):
    case = W.spd_from_spectrum(96, 0.3, 3)
    check_parity(case, p, form="literal")


def test_coupled_form_p1():
    case = W.spd_from_spectrum(128, 0.05, 4)
    check_parity(case, 1, form="coupled")


def test_host_buffers():
    case = W.spd_from_spectrum(150, 0.05, 6)
    Cd, *_rest, h = gpu_solve(case.A, 2)
    P.pr_destroy(h)
    Ch, *_rest, h = gpu_solve(case.A, 2, host=True)
    P.pr_destroy(h)
    assert np.array_equal(Cd, Ch)


def test_deterministic():
    case = W.spd_from_spectrum(200, 0.01, 7)
    a, *_r, h = gpu_solve(case.A, 3)
    P.pr_destroy(h)
    b, *_r, h = gpu_solve(case.A, 3)
    P.pr_destroy(h)
    assert np.array_equal(a, b)


def test_true_residual_matches_definition():
    case = W.spd_from_spectrum(180, 0.02, 8)
    for p in (1, 2, 3):
        C, st, steps, hist, stats, h = gpu_solve(case.A, p)
        try:
            r = P.pr_residual(h, P.PR_FP64)
        finally:
            P.pr_destroy(h)
        want = O.residual_fro(C, case.A, p)
        assert abs(r - want) <= 1e-3 * want + 1e-14, (p, r, want)


def test_stop_reasons():
    case = W.spd_from_spectrum(128, 0.01, 9)
    C, st, steps, hist, stats, h = gpu_solve(case.A, 1, tol=0.0)
    P.pr_destroy(h)
    assert st == P.PR_ESTAGNATED and hist[-2] < 1e-3
    C, st, steps, hist, stats, h = gpu_solve(case.A, 2, tol=0.0, max_iter=5)
    P.pr_destroy(h)
    assert st == P.PR_EMAXITER and steps == 5 and len(hist) == 6 and stats["iterations"] == 5


def test_resume_and_stats():
    case = W.spd_from_spectrum(128, 0.01, 10)
    o = P.pr_default_options()
    A = torch.from_numpy(case.A).to(DEV)
    h = P.pr_init(A, 128, 2, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        st1, d1 = P.pr_iterate(h, 7, P.PR_FP64, 1e-12)
        st2, d2 = P.pr_iterate(h, 100, P.PR_FP64, 1e-12)
        s = P.pr_stats(h)
    finally:
        P.pr_destroy(h)
    Co, info = O.solve(case.A, 2, tol=1e-12)
    assert st1 == P.PR_EMAXITER and d1 == 7
    # The oracle's verified stop decides between PR_OK and PR_EINACCURATE (Eq. 3's C_0 at kappa = 1e2).
    assert st2 == {"tol": P.PR_OK, "inaccurate": P.PR_EINACCURATE}[info.stop]
    assert abs(d1 + d2 - info.iterations) <= 1
    assert s["iterations"] == d1 + d2 and s["iterations_by_precision"][P.PR_FP64] == d1 + d2
    assert s["norm_1"] == pytest.approx(O.norm_1(case.A), rel=1e-14)
    assert s["norm_inf"] == pytest.approx(O.norm_inf(case.A), rel=1e-14)
    # M_0 (2 products), 3 per update, and the verification at each of the two stops (X X, then X^2 A).
    assert s["gemms"] == 2 + 3 * s["iterations"] + 2 * 2


def test_input_errors():
    stream = torch.cuda.current_stream(DEV).cuda_stream
    case = W.spd_from_spectrum(40, 0.1, 11)
    A = case.A.copy()
    A[3, 5] += 1e-3
    with pytest.raises(P.PthrootError) as e:
        P.pr_init(torch.from_numpy(A).to(DEV), 40, 2, None, stream)
    assert e.value.status == P.PR_EINVAL and "symmetric" in str(e.value)
    A = case.A.copy()
    A[2, 2] = np.nan
    with pytest.raises(P.PthrootError) as e:
        P.pr_init(torch.from_numpy(A).to(DEV), 40, 2, None, stream)
    assert e.value.status == P.PR_EINVAL
    A = case.A.copy()
    A[4, 4] = -1.0
    with pytest.raises(P.PthrootError) as e:
        P.pr_init(torch.from_numpy(A).to(DEV), 40, 2, None, stream)
    assert e.value.status == P.PR_ENOTSPD


@pytest.mark.parametrize("where", [(2, 3, 100), (70, 71, 100), (99, 97, 100)])
def test_indefinite_with_positive_diagonal(where):
    # I + 2 (e_i e_j^T + e_j e_i^T) has the eigenvalue -1 and a unit diagonal: the Cholesky factorisation of
    # the diagonal block of order 64 that holds rows i and j fails (in the first, the second and the last,
    # ragged block of an order-100 matrix).
    i, j, n = where
    A = np.eye(n)
    A[i, j] = A[j, i] = 2.0
    with pytest.raises(P.PthrootError) as e:
        P.pr_init(torch.from_numpy(A).to(DEV), n, 2, None, torch.cuda.current_stream(DEV).cuda_stream)
    assert e.value.status == P.PR_ENOTSPD and "Cholesky" in str(e.value)


def test_coupled_stop_is_verified():
    # The oracle's verified stop (Eq. 3's M_0 spans kappa^(p+1); at kappa = 1e3, p = 3 the carried
    # ||I - M||_F meets 1e-12 while the true residual stays far above it) is what the library reports:
    # PR_EINACCURATE, with the true residual of its result in the stats. Without verification: PR_OK and
    # no true residual.
    case = W.spd_from_spectrum(128, 1e-3, 5)
    Co, info = O.solve(case.A, 3, tol=1e-12)
    assert info.stop == "inaccurate"
    C, st, steps, hist, stats, h = gpu_solve(case.A, 3)
    P.pr_destroy(h)
    assert st == P.PR_EINACCURATE and hist[-1] <= 1e-12
    want = O.residual_fro(C, case.A, 3)
    assert stats["true_residual"] == pytest.approx(want, rel=1e-6) and want > 1e-9
    o = P.pr_default_options()
    o.verify = 0
    h = P.pr_init(torch.from_numpy(case.A).to(DEV), 128, 3, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        st2, _ = P.pr_iterate(h, 100, P.PR_FP64, 1e-12)
        s2 = P.pr_stats(h)
    finally:
        P.pr_destroy(h)
    assert st2 == P.PR_OK and s2["true_residual"] == -1.0
    # The scaled identity (M_0 spans kappa) meets the tolerance for real at kappa = 10.
    case = W.spd_from_spectrum(64, 0.1, 5)
    C, st, steps, hist, stats, h = gpu_solve(case.A, 3, c0="scaled_identity")
    P.pr_destroy(h)
    assert st == P.PR_OK and 0 < stats["true_residual"] <= 1e-12
    assert stats["true_residual"] == pytest.approx(O.residual_fro(C, case.A, 3), rel=1e-2, abs=1e-14)


@pytest.mark.parametrize("p", [2, 3])
def test_prescale_for_eq2(p):
    # ||A||_1 < 1 with p > 1: Eq. 3's C_0 would violate Eq. 2 (the oracle diverges on A itself); the library
    # iterates on 2^k A (the oracle's eq2_prescale reading) and returns 2^(k/p) times that root. Compared with
    # the oracle's solve of the scaled problem and with the closed form of the shrunk matrix.
    case = W.spd_from_spectrum(150, 0.05, 30 + p)
    A = 0.01 * case.A
    As, k = O.eq2_prescale(A, p)
    Co, info = O.solve(As, p, tol=1e-12)
    Co = 2.0 ** (k / p) * Co
    Z = O.closed_form_root(case.Q, 0.01 * case.lam, p)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    C, st, steps, hist, stats, h = gpu_solve(A, p)
    P.pr_destroy(h)
    assert stats["prescale_log2"] == k > 0
    assert stats["norm_1"] == pytest.approx(O.norm_1(As), rel=1e-14)
    assert O.forward_error(C, Z) <= bound and O.forward_error(C, Co) <= bound
    assert abs(steps - info.iterations) <= 1
    # p = 1 needs no scaling (Eq. 3 is scale-invariant there).
    C1, st1, _, _, stats1, h = gpu_solve(A, 1)
    P.pr_destroy(h)
    assert stats1["prescale_log2"] == 0
    assert O.forward_error(C1, O.closed_form_root(case.Q, 0.01 * case.lam, 1)) <= 1e-12


def test_p4_chain_uses_squares():
    # p = 4: M' = N^4 M is formed as (N^2)^2 M, three products per update (plus X N); M_0 = X^4 A keeps the
    # plain chain of four. Same iterates as the oracle's N (N (N (N M))) up to rounding.
    case = W.spd_from_spectrum(130, 0.05, 12)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    h = P.pr_init(torch.from_numpy(case.A).to(DEV), 130, 4, P.pr_default_options(), stream)
    try:
        st, d = P.pr_iterate(h, 100, P.PR_FP64, 1e-12)
        s = P.pr_stats(h)
        C = torch.empty((130, 130), dtype=torch.float64, device=DEV)
        P.pr_result(h, C)
    finally:
        P.pr_destroy(h)
    assert s["gemms"] == 4 + 4 * s["iterations"] + 4  # + the verification at the stop: X^4 by 3, then A
    Co, info = O.solve(case.A, 4, tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, 4)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C.cpu().numpy(), Z) <= bound and O.forward_error(C.cpu().numpy(), Co) <= bound
    assert abs(d - info.iterations) <= 1


@pytest.mark.parametrize("prec", [P.PR_FP64, P.PR_EMU64])
def test_p3_update_takes_two_products(prec):
    # p = 3: M' = N^3 M is formed as L R, L = (4M - M^2)/27, R = 16I - 8M + M^2 (two products, plus X N);
    # M_0 = X^3 A keeps the plain chain of three. Same iterates as the oracle's N (N (N M)) up to rounding.
    case = W.spd_from_spectrum(140, 0.02, 13)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    h = P.pr_init(torch.from_numpy(case.A).to(DEV), 140, 3, P.pr_default_options(), stream)
    try:
        st, d = P.pr_iterate(h, 100, prec, 1e-12)
        s = P.pr_stats(h)
        C = torch.empty((140, 140), dtype=torch.float64, device=DEV)
        P.pr_result(h, C)
    finally:
        P.pr_destroy(h)
    assert s["gemms"] == 3 + 3 * s["iterations"] + 3  # + the verification at the stop: X^3 by 2, then A
    Co, info = O.solve(case.A, 3, tol=1e-12)
    Z = O.closed_form_root(case.Q, case.lam, 3)
    bound = max(1e-12, 10 * O.forward_error(Co, Z))
    assert O.forward_error(C.cpu().numpy(), Z) <= bound and O.forward_error(C.cpu().numpy(), Co) <= bound
    assert abs(d - info.iterations) <= 1


def test_bounded_wait_expires_and_context_survives():
    # A device wait that nothing completes runs out after its limit and is reported as PR_ETIMEOUT; the
    # next products on the same context are still correct.
    st, waited = P.pr_selftest_wait(torch.cuda.current_stream(DEV).cuda_stream)
    assert st == P.PR_ETIMEOUT and 1.9 < waited < 3.0
    assert "expected" in P.pr_last_error()
    case = W.spd_from_spectrum(130, 0.05, 12)
    X = torch.from_numpy(case.A).to(DEV)
    Pd = torch.empty_like(X)
    P.pr_matmul(P.PR_EMU64, X, X, 130, True, Pd, torch.cuda.current_stream(DEV).cuda_stream)
    np.testing.assert_allclose(Pd.cpu().numpy(), case.A @ case.A, rtol=1e-12, atol=1e-14)
