"""Newton refinement of an approximate root (pr_refine, pr_set_iterate), through the C ABI.

Parity: from the same perturbed root, the GPU refinement with FP64-accurate products (PR_EMU64 for the
residual and the solve) follows the oracle's refine_newton step by step: the same residuals while they are far
above rounding, about the same conjugate-gradient lengths, and a result within max(1e-12, 10 x the oracle's
forward error) of the closed form. With low-precision solves (PR_FP32X, PR_BF16) each step gains less, and the
result after more steps meets the same bar. From the library's own Eq. 3 solves, whose coupled form loses
u kappa^(p+1), refinement reaches FP64 accuracy. Orders span several 128 x 96 tiles with ragged tails.
"""
import ctypes

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


def stream():
    return torch.cuda.current_stream(DEV).cuda_stream


def perturbed_root(n, lam_min, seed, p, rel=1e-3):
    c = W.spd_from_spectrum(n, lam_min, seed)
    Z = O.closed_form_root(c.Q, c.lam, p)
    X0 = np.ascontiguousarray(Z + rel * np.linalg.norm(Z) * W.symmetric_perturbation(n, seed + 1000))
    return c, Z, X0


def refine_on_gpu(A, X0, p, prec, inner, max_steps, tol, cg_max, cg_tol, options=None):
    n = A.shape[0]
    h = P.pr_init(torch.from_numpy(A).to(DEV), n, p, options, stream())
    try:
        P.pr_set_iterate(h, torch.from_numpy(X0).to(DEV))
        st, k = P.pr_refine(h, prec, inner, max_steps, tol, cg_max, cg_tol)
        C = torch.empty((n, n), dtype=torch.float64, device=DEV)
        P.pr_result(h, C)
        stats = P.pr_stats(h)
    finally:
        P.pr_destroy(h)
    return C.cpu().numpy(), st, k, stats


@pytest.mark.parametrize("n", [100, 257])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_refinement_follows_the_oracle(n, p):
    c, Z, X0 = perturbed_root(n, 1e-2, 70 + n + p, p)
    cg_tol = 1e-10
    C, st, k, stats = refine_on_gpu(c.A, X0, p, P.PR_EMU64, P.PR_EMU64, 3, 0.0, 60, cg_tol)
    Xo, info = O.refine_newton(c.A, X0, p, max_steps=3, tol=0.0, cg_max=60, cg_tol=cg_tol)
    hg, ho = np.asarray(stats["refine_residuals"]), np.asarray(info.residuals)
    assert len(hg) >= 2 and len(ho) >= 2
    # the residual of the common start, evaluated with FP64-accurate products on both sides
    assert hg[0] == pytest.approx(ho[0], rel=1e-10)
    # later residuals: equal while far above rounding (the solves agree to about cg_tol)
    m = min(len(hg), len(ho))
    far = [i for i in range(1, m) if ho[i] > 1e-9]
    np.testing.assert_allclose(hg[far], ho[far], rtol=1e-3)
    for a, b in zip(stats["refine_cg"], info.cg_iterations):
        assert abs(a - b) <= 3
    bar = max(1e-12, 10 * O.forward_error(Xo, Z))
    assert O.forward_error(C, Z) <= bar
    assert O.forward_error(C, Xo) <= bar
    assert np.array_equal(C, C.T)
    # the reported true residual is that of the returned root (at the rounding floor, up to rounding)
    assert stats["true_residual"] == pytest.approx(O.residual_fro(C, c.A, p), rel=1e-2, abs=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_native_fp64_products_follow_the_oracle(p):
    # The residual and the solve with native FP64 (DMMA) products, whose kernel computes X Y (not X Y^T): the
    # p = 3 residual takes the W V form there.
    c, Z, X0 = perturbed_root(200, 1e-2, 150 + p, p)
    C, st, k, stats = refine_on_gpu(c.A, X0, p, P.PR_FP64, P.PR_FP64, 3, 0.0, 60, 1e-10)
    Xo, info = O.refine_newton(c.A, X0, p, max_steps=3, tol=0.0, cg_max=60, cg_tol=1e-10)
    hg, ho = np.asarray(stats["refine_residuals"]), np.asarray(info.residuals)
    assert hg[0] == pytest.approx(ho[0], rel=1e-10)
    m = min(len(hg), len(ho))
    far = [i for i in range(1, m) if ho[i] > 1e-9]
    np.testing.assert_allclose(hg[far], ho[far], rtol=1e-3)
    assert O.forward_error(C, Z) <= max(1e-12, 10 * O.forward_error(Xo, Z))


def test_start_outside_the_region_of_convergence_is_left_unchanged():
    # Eq. 3's C_0 is far from the root for p = 2 at kappa = 1e2: a correction that does not lower the residual
    # is undone, and the handle keeps the iterate it was given.
    n, p = 160, 2
    c = W.spd_from_spectrum(n, 1e-2, 61)
    X0 = np.ascontiguousarray(O.initial_guess_eq3(c.A))
    Xo, info = O.refine_newton(c.A, X0, p, max_steps=4, tol=0.0)
    C, st, k, stats = refine_on_gpu(c.A, X0, p, P.PR_EMU64, P.PR_EMU64, 4, 0.0, 50, 1e-12)
    assert st in (P.PR_ESTAGNATED, P.PR_EMAXITER, P.PR_EDIVERGED)
    r = stats["refine_residuals"]
    assert all(b < a for a, b in zip(r, r[1:]))  # every kept step lowered the residual
    if info.steps == 0:  # the oracle keeps the start too: so must the library
        assert k == 0 and np.array_equal(C, X0)


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("inner,cg_tol,steps", [(P.PR_FP32X, 1e-6, 6), (P.PR_BF16, 1e-2, 12)])
def test_low_precision_solves_reach_the_bar(p, inner, cg_tol, steps):
    n = 300
    c, Z, X0 = perturbed_root(n, 1e-2, 90 + p, p)
    C, st, k, stats = refine_on_gpu(c.A, X0, p, P.PR_EMU64, inner, steps, 0.0, 80, cg_tol)
    Xo, _ = O.refine_newton(c.A, X0, p, max_steps=6, tol=0.0)
    assert O.forward_error(C, Z) <= max(1e-12, 10 * O.forward_error(Xo, Z)), stats["refine_residuals"]
    assert st in (P.PR_ESTAGNATED, P.PR_EMAXITER)
    # every kept step lowered the residual
    r = stats["refine_residuals"]
    assert all(b < a for a, b in zip(r, r[1:]))


def test_fp8_solves_still_improve_the_root():
    n, p = 200, 2
    c, Z, X0 = perturbed_root(n, 1e-2, 97, p)
    C, st, k, stats = refine_on_gpu(c.A, X0, p, P.PR_EMU64, P.PR_FP8, 4, 0.0, 20, 0.1)
    assert k >= 1 and O.forward_error(C, Z) < 0.1 * O.forward_error(X0, Z)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_eq3_solves_refined_to_fp64_accuracy(p):
    # The coupled form from Eq. 3's C_0 at kappa = 1e3 ends far from FP64 accuracy (u kappa^(p+1)); a few
    # corrections with split-FP32 solves bring it to the accuracy of the oracle from the scaled identity.
    n = 512
    c = W.spd_from_spectrum(n, 1e-3, 31)
    Z = O.closed_form_root(c.Q, c.lam, p)
    h = P.pr_init(torch.from_numpy(c.A).to(DEV), n, p, None, stream())
    try:
        P.pr_iterate(h, 100, P.PR_EMU64, 1e-12)
        C0 = torch.empty((n, n), dtype=torch.float64, device=DEV)
        P.pr_result(h, C0)
        st, k = P.pr_refine(h, P.PR_EMU64, P.PR_FP32X, 8, 0.0, 80, 1e-6)
        C = torch.empty((n, n), dtype=torch.float64, device=DEV)
        P.pr_result(h, C)
        stats = P.pr_stats(h)
        # Eq. 1 may continue after a refinement (M is re-formed from the refined X)
        st2, _ = P.pr_iterate(h, 3, P.PR_EMU64, 1e-12)
        C2 = torch.empty((n, n), dtype=torch.float64, device=DEV)
        P.pr_result(h, C2)
    finally:
        P.pr_destroy(h)
    before, after = O.forward_error(C0.cpu().numpy(), Z), O.forward_error(C.cpu().numpy(), Z)
    Xs, _ = O.solve(c.A, p, c0="scaled_identity", tol=1e-12)
    bar = max(1e-12, 10 * O.forward_error(Xs, Z))
    assert before > 1e-10
    assert after <= bar, (before, after, stats["refine_residuals"], stats["refine_cg"])
    assert 1 <= k <= 8 and st == P.PR_ESTAGNATED
    assert O.forward_error(C2.cpu().numpy(), Z) <= bar


def test_tiny_orders():
    for n, p in ((1, 2), (1, 3), (17, 4), (17, 1)):
        c, Z, X0 = perturbed_root(n, 0.1, 5 + n, p, rel=1e-2)
        C, st, k, stats = refine_on_gpu(c.A, X0, p, P.PR_EMU64, P.PR_EMU64, 6, 0.0, 40, 1e-12)
        assert O.forward_error(C, Z) < 1e-13, (n, p, stats["refine_residuals"])


def test_prescaled_matrix_and_set_iterate_round_trip():
    # ||A||_1 < 1 with p = 2: the handle iterates on 2^k A (Eq. 2); pr_set_iterate takes and pr_result gives
    # roots of the caller's A.
    n, p = 150, 2
    c = W.spd_from_spectrum(n, 1e-2, 44)
    A = np.ascontiguousarray(0.01 * c.A)
    Z = O.closed_form_root(c.Q, 0.01 * c.lam, p)
    X0 = np.ascontiguousarray(Z + 1e-3 * np.linalg.norm(Z) * W.symmetric_perturbation(n, 45))
    h = P.pr_init(torch.from_numpy(A).to(DEV), n, p, None, stream())
    try:
        assert P.pr_stats(h)["prescale_log2"] != 0
        P.pr_set_iterate(h, torch.from_numpy(X0).to(DEV))
        back = torch.empty((n, n), dtype=torch.float64, device=DEV)
        P.pr_result(h, back)
        np.testing.assert_allclose(back.cpu().numpy(), X0, rtol=5e-16, atol=0)
        st, k = P.pr_refine(h, P.PR_EMU64, P.PR_FP32X, 6, 0.0, 60, 1e-6)
        P.pr_result(h, back)
    finally:
        P.pr_destroy(h)
    assert O.forward_error(back.cpu().numpy(), Z) < 1e-13


def test_errors():
    n = 64
    c = W.spd_from_spectrum(n, 0.1, 3)
    A = torch.from_numpy(c.A).to(DEV)
    h = P.pr_init(A, n, 2, None, stream())
    L = P._lib
    try:
        C0 = torch.empty((n, n), dtype=torch.float64, device=DEV)
        P.pr_result(h, C0)
        C_before = C0.cpu().numpy()
        for args in ((P.PR_EMU64, 99, 2, 0.0, 10, 1e-6), (7, P.PR_EMU64, 2, 0.0, 10, 1e-6),
                     (P.PR_EMU64, P.PR_EMU64, P.PR_REFINE_MAX_STEPS + 1, 0.0, 10, 1e-6),
                     (P.PR_EMU64, P.PR_EMU64, -1, 0.0, 10, 1e-6), (P.PR_EMU64, P.PR_EMU64, 2, -1.0, 10, 1e-6),
                     (P.PR_EMU64, P.PR_EMU64, 2, 0.0, 0, 1e-6), (P.PR_EMU64, P.PR_EMU64, 2, 0.0, 10, float("nan"))):
            assert L.pr_refine(h, *args, None) == P.PR_EINVAL, args
        bad = c.A.copy()
        bad[3, 5] = np.nan
        assert L.pr_set_iterate(h, ctypes.c_void_p(torch.from_numpy(bad).to(DEV).data_ptr())) == P.PR_EINVAL
        bad = c.A.copy()
        bad[3, 5] += 1e-3
        assert L.pr_set_iterate(h, ctypes.c_void_p(torch.from_numpy(bad).to(DEV).data_ptr())) == P.PR_EINVAL
        bad = -np.eye(n)
        assert L.pr_set_iterate(h, ctypes.c_void_p(torch.from_numpy(bad).to(DEV).data_ptr())) == P.PR_ENOTSPD
        assert L.pr_set_iterate(h, None) == P.PR_EINVAL
        # the refused iterates left the handle as it was: Eq. 3's C_0, untouched
        C = torch.empty((n, n), dtype=torch.float64, device=DEV)
        P.pr_result(h, C)
        np.testing.assert_array_equal(C.cpu().numpy(), C_before)
    finally:
        P.pr_destroy(h)
    assert L.pr_refine(None, P.PR_EMU64, P.PR_EMU64, 1, 0.0, 10, 1e-6, None) == P.PR_ESTATE
    h = P.pr_init(A, n, 5, None, stream())
    try:
        assert L.pr_refine(h, P.PR_EMU64, P.PR_EMU64, 1, 0.0, 10, 1e-6, None) == P.PR_EUNSUPPORTED
    finally:
        P.pr_destroy(h)


def test_exact_root_stops_at_once():
    n, p = 120, 3
    c = W.spd_from_spectrum(n, 0.1, 8)
    Z = O.closed_form_root(c.Q, c.lam, p)
    C, st, k, stats = refine_on_gpu(c.A, Z, p, P.PR_EMU64, P.PR_FP32X, 4, 1e-10, 40, 1e-6)
    assert st == P.PR_OK and k == 0 and stats["refine_len"] == 1
    np.testing.assert_array_equal(C, Z)
