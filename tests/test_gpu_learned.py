"""The learned polynomial initial guess on the GPU, through the C ABI: features, the gated polynomial
C_0, the device MLP against the CPU oracle MLP, and what the trained network gains over the plain method."""
import numpy as np
import pytest

from oracle import pthroot_oracle as O
from paper_1703_02283_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1703_02283_gb300 import learned as L  # noqa: E402
from paper_1703_02283_gb300 import pthroot as P  # noqa: E402

DEV = torch.device("cuda:0")


def handle(S, p, **opt):
    o = P.pr_default_options()
    for k, v in opt.items():
        if k == "c0_coef":
            for i in range(4):
                o.c0_coef[i] = float(v[i])
        else:
            setattr(o, k, v)
    return P.pr_init(torch.from_numpy(S).to(DEV), S.shape[0], p, o, torch.cuda.current_stream(DEV).cuda_stream)


def test_features_match_oracle():
    for n, seed in ((96, 1), (300, 2)):
        c = W.spd_from_spectrum(n, 0.02, seed)
        h = handle(c.A, 2)
        try:
            f = np.array(P.pr_features(h))
        finally:
            P.pr_destroy(h)
        np.testing.assert_allclose(f, O.spectral_features(c.A), rtol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_polynomial_guess_matches_oracle_and_gate(p):
    # Fit on [lambda_min, 1.1 lambda_max] / ||A||_1: q then stays positive past the 5 % margin the library
    # checks above its estimate of ||A||_2 (first zero of q at >= 1.11 lambda_max / ||A||_1 for these cases).
    c = W.spd_from_spectrum(200, 1e-2, 30 + p)
    s = O.norm_1(c.A)
    coef = O.relative_fit(c.lam.min() / s, 1.1 * c.lam.max() / s, p)
    h = handle(c.A, p, c0=P.PR_C0_POLY, c0_coef=coef)
    try:
        st = P.pr_stats(h)
        P.pr_iterate(h, 0, P.PR_FP64, 0.0)  # no update: the current iterate is C_0
        C0 = torch.empty((200, 200), dtype=torch.float64, device=DEV)
        P.pr_result(h, C0)
    finally:
        P.pr_destroy(h)
    want = O.polynomial_initial_guess(c.A, p, coef)
    g = O.gate_value(c.A, p, want)  # exact ||I - C_0^p A||_2, below 0.85 for these cases
    assert g < 0.85
    assert st["c0"] == P.PR_C0_POLY
    np.testing.assert_allclose(C0.cpu().numpy(), want, rtol=1e-11, atol=1e-14)
    # The power iteration approaches ||I - C_0^p A||_2 from below.
    assert 0.9 * g <= st["c0_gate"] <= g * (1 + 1e-9)


def test_polynomial_negative_past_spectrum_falls_back():
    # The p = 1 fit on exactly [lambda_min, lambda_max] / ||A||_1 has a zero at 1.016 lambda_max / ||A||_1,
    # inside the checked margin: C_0 would be fine on this spectrum but the guess is refused (gate = inf).
    c = W.spd_from_spectrum(200, 1e-2, 31)
    s = O.norm_1(c.A)
    coef = O.relative_fit(c.lam.min() / s, c.lam.max() / s, 1)
    h = handle(c.A, 1, c0=P.PR_C0_POLY, c0_coef=coef)
    try:
        st = P.pr_stats(h)
        P.pr_iterate(h, 0, P.PR_FP64, 0.0)
        C0 = torch.empty((200, 200), dtype=torch.float64, device=DEV)
        P.pr_result(h, C0)
    finally:
        P.pr_destroy(h)
    assert st["c0"] == P.PR_C0_EQ3 and st["c0_gate"] == float("inf")
    np.testing.assert_allclose(C0.cpu().numpy(), O.initial_guess_eq3(c.A), rtol=1e-13, atol=1e-18)


def test_set_initial_guess_matches_fresh_handles():
    # Features -> pr_set_initial_guess on one handle must give, bit for bit, what a handle created with the
    # same polynomial gives (the cached A^2, A^3 are the same products); switching back to Eq. 3 restarts
    # from Eq. 3's C_0; a later pr_load forms C_0 as pr_init's options say.
    c = W.spd_from_spectrum(160, 1e-2, 50)
    s = O.norm_1(c.A)
    coef = O.relative_fit(c.lam.min() / s, 1.1 * c.lam.max() / s, 2)

    def run(h):
        P.pr_iterate(h, 100, P.PR_EMU64, 1e-12)
        C = torch.empty((160, 160), dtype=torch.float64, device=DEV)
        P.pr_result(h, C)
        return C.cpu().numpy(), P.pr_history(h), P.pr_stats(h)

    hp = handle(c.A, 2, c0=P.PR_C0_POLY, c0_coef=coef)
    he = handle(c.A, 2)
    h = handle(c.A, 2)
    try:
        Cp, hist_p, st_p = run(hp)
        Ce, hist_e, _ = run(he)
        f = P.pr_features(h)
        np.testing.assert_allclose(f, O.spectral_features(c.A), rtol=1e-12)
        P.pr_set_initial_guess(h, P.PR_C0_POLY, coef)
        C1, hist_1, st_1 = run(h)
        assert st_1["c0"] == P.PR_C0_POLY and st_1["c0_gate"] == st_p["c0_gate"]
        assert np.array_equal(C1, Cp) and hist_1 == hist_p and st_1["iterations"] == st_p["iterations"]
        P.pr_set_initial_guess(h, P.PR_C0_EQ3)
        C0 = torch.empty((160, 160), dtype=torch.float64, device=DEV)
        P.pr_result(h, C0)
        np.testing.assert_allclose(C0.cpu().numpy(), O.initial_guess_eq3(c.A), rtol=1e-13, atol=1e-18)
        C2, hist_2, _ = run(h)
        assert np.array_equal(C2, Ce) and hist_2 == hist_e
        P.pr_set_initial_guess(h, P.PR_C0_POLY, coef)
        P.pr_load(h, torch.from_numpy(c.A).to(DEV))
        assert P.pr_stats(h)["c0"] == P.PR_C0_EQ3
        with pytest.raises(P.PthrootError) as e:
            P.pr_set_initial_guess(h, 7)
        assert e.value.status == P.PR_EINVAL
        with pytest.raises(P.PthrootError) as e:
            P.pr_set_initial_guess(h, P.PR_C0_POLY, None)
        assert e.value.status == P.PR_EINVAL
        with pytest.raises(P.PthrootError) as e:
            P.pr_set_initial_guess(h, P.PR_C0_POLY, [1.0, float("nan"), 0.0, 0.0])
        assert e.value.status == P.PR_EINVAL
    finally:
        for x in (hp, he, h):
            P.pr_destroy(x)
    assert Cp.shape == (160, 160)


def test_gate_falls_back_to_eq3():
    c = W.spd_from_spectrum(128, 1e-2, 40)
    for coef in ([1.0, -3.0, 0.0, 0.0],  # q < 0 on [0, 1]
                 [40.0, 0.0, 0.0, 0.0]):  # positive but ||I - C_0^2 A|| far above 1
        h = handle(c.A, 2, c0=P.PR_C0_POLY, c0_coef=coef)
        try:
            st = P.pr_stats(h)
            P.pr_iterate(h, 100, P.PR_EMU64, 1e-12)
            C = torch.empty((128, 128), dtype=torch.float64, device=DEV)
            P.pr_result(h, C)
        finally:
            P.pr_destroy(h)
        assert st["c0"] == P.PR_C0_EQ3
        Z = O.closed_form_root(c.Q, c.lam, 2)
        Co, _ = O.solve(c.A, 2, tol=1e-12)
        assert O.forward_error(C.cpu().numpy(), Z) <= max(1e-12, 10 * O.forward_error(Co, Z))


def test_mlp_forward_and_gradient_match_oracle():
    rng = np.random.default_rng(3)
    theta = L.init_params(7)
    X = rng.standard_normal((200, 8)).astype(np.float32)
    T = rng.standard_normal((200, 4)).astype(np.float32)
    m = P.pr_mlp_create(theta, 200)
    try:
        Y = np.empty((200, 4), dtype=np.float32)
        P.pr_mlp_forward(m, X, 200, Y)
        g = np.empty(P.PR_MLP_PARAMS, dtype=np.float32)
        loss = P.pr_mlp_loss_grad(m, X, T, 200, g)
    finally:
        P.pr_mlp_destroy(m)
    Yo = O.mlp_forward(theta.astype(np.float64), X.astype(np.float64))
    lo, go = O.mlp_loss_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    np.testing.assert_allclose(Y, Yo, rtol=1e-4, atol=1e-5)
    assert loss == pytest.approx(lo, rel=1e-5)
    # FP32 against FP64: relative to the gradient's scale
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go) + 1e-7


def test_adam_training_decreases_loss_and_is_deterministic():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((256, 8)).astype(np.float32)
    T = np.tanh(X[:, :4] @ rng.standard_normal((4, 4))).astype(np.float32)
    runs = []
    for _ in range(2):
        m = P.pr_mlp_create(L.init_params(1), 256)
        try:
            losses = [P.pr_mlp_adam_step(m, X, T, 256, 1e-2) for _ in range(150)]
            th = np.empty(P.PR_MLP_PARAMS, dtype=np.float32)
            P.pr_mlp_get_params(m, th)
        finally:
            P.pr_mlp_destroy(m)
        runs.append((losses, th))
    assert runs[0][0][-1] < 0.2 * runs[0][0][0]
    assert np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.slow
def test_trained_network_cuts_iterations():
    # Small version of the drifting-overlap workload: n = 256, 6 training sequences x 6 samples, 2 test
    # sequences. The network's guess must pass the gate and cut iterations against Eq. 3, with FP64-level
    # accuracy.
    n, p = 256, 2
    stream = torch.cuda.current_stream(DEV).cuda_stream
    train = [S for s in range(6) for S in L.overlap_sequence(s, 30, n, every=5)]
    test = [S for s in (40, 41) for S in L.overlap_sequence(s, 30, n, every=10)]
    samples = L.make_samples(torch, train, p, stream)
    model = L.train(samples, steps=600, lr=3e-3, stream=stream)
    assert model.loss_history[-1] < 0.1 * model.loss_history[0]
    tests = L.make_samples(torch, test, p, stream)
    coefs = L.predict(model, np.stack([t.features for t in tests]), stream)
    gained = 0
    for S, t, c in zip(test, tests, coefs):
        C, its, used, gate = L.solve_with_guess(torch, S, p, c, stream=stream)
        Z = O.eig_root(S, p)
        assert O.forward_error(C, Z) < 1e-12
        if used == P.PR_C0_POLY:
            gained += t.iterations - its
            assert its < t.iterations
    assert gained > 0


def test_gate_without_fallback_reports_egate():
    # gate_fallback = 0: a guess that fails the gate is an error (PR_EGATE) instead of a silent fallback.
    # pr_init creates no handle; pr_set_initial_guess leaves Eq. 3's C_0 in the handle, which still solves.
    c = W.spd_from_spectrum(128, 1e-2, 40)
    bad = [40.0, 0.0, 0.0, 0.0]  # positive, but ||I - C_0^2 A||_2 far above 1
    with pytest.raises(P.PthrootError) as e:
        handle(c.A, 2, c0=P.PR_C0_POLY, c0_coef=bad, gate_fallback=0)
    assert e.value.status == P.PR_EGATE
    h = handle(c.A, 2, gate_fallback=0)
    try:
        with pytest.raises(P.PthrootError) as e:
            P.pr_set_initial_guess(h, P.PR_C0_POLY, bad)
        assert e.value.status == P.PR_EGATE and "gate" in str(e.value)
        st = P.pr_stats(h)
        assert st["c0"] == P.PR_C0_EQ3 and st["c0_gate"] > 0.9
        P.pr_iterate(h, 100, P.PR_EMU64, 1e-12)
        C = torch.empty((128, 128), dtype=torch.float64, device=DEV)
        P.pr_result(h, C)
    finally:
        P.pr_destroy(h)
    Z = O.closed_form_root(c.Q, c.lam, 2)
    Co, _ = O.solve(c.A, 2, tol=1e-12)
    assert O.forward_error(C.cpu().numpy(), Z) <= max(1e-12, 10 * O.forward_error(Co, Z))


def test_spectral_bounds_from_the_device():
    # pr_spectral_bounds: power iterations on A (||A||_2 = lambda_max = 1 for this recipe) and on the
    # converged root (||C||_2^(-p) = lambda_min), both from below / above as power iteration gives them; a
    # scaled A (p > 1, ||A||_1 < 1, iterated as 2^k A) reports the caller's eigenvalues.
    c = W.spd_from_spectrum(200, 1e-2, 41)
    for scale, p in ((1.0, 2), (0.01, 2), (1.0, 1)):
        h = handle(scale * c.A, p)
        try:
            P.pr_iterate(h, 100, P.PR_EMU64, 1e-12)
            lo, hi = P.pr_spectral_bounds(h, 80)
        finally:
            P.pr_destroy(h)
        assert 0.95 * scale <= hi <= scale * (1 + 1e-12), (scale, p, hi)
        assert scale * 1e-2 * (1 - 1e-9) <= lo <= 1.05 * scale * 1e-2, (scale, p, lo)
