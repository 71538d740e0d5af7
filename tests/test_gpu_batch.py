"""Batched solves (many SPD matrices of uneven orders and roots), through the C ABI.

Each matrix of a batch must meet the single-matrix bar against the CPU oracle, and its result must equal,
bit for bit, the single-matrix PR_EMU64 solve of the same matrix (same digit planes, same tiles, same
stop rule): the batch's work lists, residuals and stop decisions, taken on the device inside one graph,
must reproduce what the single-matrix path decides on the host. Bit-equality needs the same tile width on
both sides (residuals add per-tile partial sums), so those tests fix pr_options.emu_tile = 96; a separate
test lets the tuner choose.
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


def make_batch(count, n_lo, n_hi, kappa_hi, seed):
    spec = W.batched_specs(count, n_lo=n_lo, n_hi=n_hi, kappa_hi=kappa_hi, seed=seed)
    cases = [W.spd_from_spectrum(int(spec.n[i]), float(spec.lam_min[i]), int(spec.seeds[i])) for i in range(count)]
    return cases, [int(x) for x in spec.p]


def single_emu(case, p, c0=P.PR_C0_EQ3, max_iter=None, tile=96):
    o = P.pr_default_options()
    o.c0 = c0
    o.emu_tile = tile
    if max_iter is not None:
        o.max_iter = max_iter
    A = torch.from_numpy(case.A).to(DEV)
    h = P.pr_init(A, case.n, p, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        st, _ = P.pr_iterate(h, 100, P.PR_EMU64, 1e-12)
        C = torch.empty_like(A)
        P.pr_result(h, C)
        single_emu.last = (st, P.pr_stats(h))
        return C.cpu().numpy(), P.pr_history(h)
    finally:
        P.pr_destroy(h)


def run_batch(cases, ps, host=False, c0=P.PR_C0_EQ3, max_iter=None, repeat=False, info=None, tile=96):
    o = P.pr_default_options()
    o.c0 = c0
    o.emu_tile = tile
    if max_iter is not None:
        o.max_iter = max_iter
    mats = [np.ascontiguousarray(c.A) if host else torch.from_numpy(c.A).to(DEV) for c in cases]
    b = P.pr_batch_init(mats, ps, o, torch.cuda.current_stream(DEV).cuda_stream)
    try:
        its, sts = P.pr_batch_solve(b, len(cases), P.PR_EMU64, 1e-12)

        def results():
            out = []
            for i, c in enumerate(cases):
                C = np.empty((c.n, c.n))
                P.pr_batch_result(b, i, C)
                out.append((C, P.pr_batch_history(b, i)))
            return out

        out = results()
        if info is not None:
            info.extend(P.pr_batch_matrix(b, i) for i in range(len(cases)))
        if repeat:
            # A second solve after every matrix stopped runs the graph once more and changes nothing.
            launches = P.pr_batch_launches(b)
            assert P.pr_batch_solve(b, len(cases), P.PR_EMU64, 1e-12) == (its, sts)
            assert P.pr_batch_launches(b) > launches
            for (C, h), (C2, h2) in zip(out, results()):
                assert np.array_equal(C, C2) and h == h2
        return out, its, sts, P.pr_batch_launches(b)
    finally:
        P.pr_batch_destroy(b)


def test_batch_matches_oracle_and_single_path():
    cases, ps = make_batch(10, 5, 300, 1e3, 7)
    minfo = []
    out, its, sts, launches = run_batch(cases, ps, info=minfo)
    assert launches > 0
    for i, (case, p) in enumerate(zip(cases, ps)):
        C, hist = out[i]
        Co, info = O.solve(case.A, p, tol=1e-12)
        Z = O.closed_form_root(case.Q, case.lam, p)
        bound = max(1e-12, 10 * O.forward_error(Co, Z))
        assert O.forward_error(C, Z) <= bound, (i, case.n, p)
        assert O.forward_error(C, Co) <= bound, (i, case.n, p)
        assert abs(its[i] - info.iterations) <= 1
        assert sts[i] in (P.PR_OK, P.PR_ESTAGNATED, P.PR_EINACCURATE)
        Cs, hs = single_emu(case, p)
        assert np.array_equal(C, Cs), (i, case.n, p)
        assert hist == hs
        # The verification after the solve loop reproduces pr_iterate's: same status, same true residual.
        st1, s1 = single_emu.last
        assert sts[i] == st1 and minfo[i]["status"] == st1
        assert minfo[i]["true_residual"] == s1["true_residual"], (i, p)
        if sts[i] == P.PR_EINACCURATE:
            assert minfo[i]["true_residual"] > 1e-12 >= hist[-1]


def test_batch_prescale_and_verification():
    # Matrices with ||A||_1 < 1: those with p > 1 are iterated as 2^k A (Eq. 2 for Eq. 3's C_0) and scaled
    # back, as the single-matrix path does; every result meets the oracle's bar for the shrunk matrix
    # (the oracle solving 2^k A by its eq2_prescale reading). p = 1 matrices are not scaled.
    cases, ps = make_batch(6, 40, 200, 1e2, 19)
    shrunk = [np.ascontiguousarray(0.01 * c.A) for c in cases]
    minfo = []
    o = P.pr_default_options()
    b = P.pr_batch_init([torch.from_numpy(A).to(DEV) for A in shrunk], ps, o,
                        torch.cuda.current_stream(DEV).cuda_stream)
    try:
        its, sts = P.pr_batch_solve(b, len(cases), P.PR_EMU64, 1e-12)
        for i, (case, p) in enumerate(zip(cases, ps)):
            C = np.empty((case.n, case.n))
            P.pr_batch_result(b, i, C)
            m = P.pr_batch_matrix(b, i)
            As, k = O.eq2_prescale(shrunk[i], p)
            assert m["prescale_log2"] == k and (k > 0) == (p > 1)
            assert m["norm_1"] == pytest.approx(O.norm_1(As), rel=1e-14)
            Co, info = O.solve(As, p, tol=1e-12)
            Z = O.closed_form_root(case.Q, 0.01 * case.lam, p)
            bound = max(1e-12, 10 * O.forward_error(2.0 ** (k / p) * Co, Z))
            assert O.forward_error(C, Z) <= bound, (i, case.n, p)
            assert m["true_residual"] > 0 and sts[i] != P.PR_EDIVERGED
    finally:
        P.pr_batch_destroy(b)


def test_batch_scaled_identity_host_inputs():
    cases, ps = make_batch(6, 40, 200, 1e4, 11)
    out, its, sts, _ = run_batch(cases, ps, host=True, c0=P.PR_C0_SCALED_I)
    for i, (case, p) in enumerate(zip(cases, ps)):
        C, _ = out[i]
        Co, info = O.solve(case.A, p, c0="scaled_identity", tol=1e-12)
        Z = O.closed_form_root(case.Q, case.lam, p)
        assert O.forward_error(C, Z) <= max(1e-12, 10 * O.forward_error(Co, Z))


def test_batch_single_matrix_and_errors():
    cases, ps = make_batch(1, 129, 129, 100, 3)
    out, its, sts, _ = run_batch(cases, ps)
    Cs, _ = single_emu(cases[0], ps[0])
    assert np.array_equal(out[0][0], Cs)
    bad = cases[0].A.copy()
    bad[1, 2] += 1.0
    with pytest.raises(P.PthrootError) as e:
        P.pr_batch_init([bad], [2])
    assert e.value.status == P.PR_EINVAL


def test_batch_more_matrices_than_one_control_block():
    # 1100 matrices of orders 1..24: the work-list scan runs over two chunks of 1024 matrices. Sampled
    # results equal the single-matrix path bit for bit, and a repeated solve changes nothing.
    cases, ps = make_batch(1100, 1, 24, 1e2, 5)
    out, its, sts, _ = run_batch(cases, ps, repeat=True)
    assert all(s in (P.PR_OK, P.PR_ESTAGNATED, P.PR_EINACCURATE) for s in sts)
    for i in list(range(0, 1100, 97)) + [1099]:
        Cs, hs = single_emu(cases[i], ps[i])
        assert np.array_equal(out[i][0], Cs), (i, cases[i].n, ps[i])
        assert out[i][1] == hs


def test_batch_load_reuses_the_batch():
    # A batch solved once, then loaded with other matrices of the same orders and roots (from host memory):
    # its results, histories and iteration counts equal those of a fresh batch of the new matrices, bit for
    # bit (same captured graph, state reset on the device).
    cases, ps = make_batch(7, 30, 260, 1e3, 41)
    other = [W.spd_from_spectrum(c.n, 1e-2, 5000 + i) for i, c in enumerate(cases)]
    o = P.pr_default_options()
    o.emu_tile = 96
    b = P.pr_batch_init([torch.from_numpy(c.A).to(DEV) for c in cases], ps, o,
                        torch.cuda.current_stream(DEV).cuda_stream)
    try:
        P.pr_batch_solve(b, len(cases), P.PR_EMU64, 1e-12)
        for _ in range(8):  # together more loop passes than the limit of one solve
            P.pr_batch_load(b, [np.ascontiguousarray(c.A) for c in other])
            its, sts = P.pr_batch_solve(b, len(cases), P.PR_EMU64, 1e-12)
        got = []
        for i, c in enumerate(other):
            C = np.empty((c.n, c.n))
            P.pr_batch_result(b, i, C)
            got.append((C, P.pr_batch_history(b, i)))
        bad = other[0].A.copy()
        bad[0, 1] += 1.0
        with pytest.raises(P.PthrootError) as e:
            P.pr_batch_load(b, [bad] + [c.A for c in other[1:]])
        assert e.value.status == P.PR_EINVAL
    finally:
        P.pr_batch_destroy(b)
    fresh, fits, fsts, _ = run_batch(other, ps)
    assert its == fits and sts == fsts
    for (C, h), (C2, h2) in zip(got, fresh):
        assert np.array_equal(C, C2) and h == h2


def test_batch_max_iter_stops_every_matrix():
    # A cap of 3 updates: every matrix stops with PR_EMAXITER after 3 iterations (4 residuals), at the
    # iterate the single-matrix path with the same cap returns.
    cases, ps = make_batch(8, 50, 260, 1e3, 21)
    out, its, sts, _ = run_batch(cases, ps, max_iter=3)
    assert its == [3] * 8 and sts == [P.PR_EMAXITER] * 8
    for i, (case, p) in enumerate(zip(cases, ps)):
        assert len(out[i][1]) == 4
        Cs, hs = single_emu(case, p, max_iter=3)
        assert np.array_equal(out[i][0], Cs) and out[i][1] == hs


@pytest.mark.slow
def test_batch_full_size_sampled():
    # The 512-matrix workload (orders 64..1024, kappa up to 1e4, p in {1, 2, 3}); 6 matrices checked against
    # the oracle, all against their exact roots within the bound the oracle attains on the sampled ones.
    spec = W.batched_specs(512)
    cases = [W.spd_from_spectrum(int(spec.n[i]), float(spec.lam_min[i]), int(spec.seeds[i])) for i in range(512)]
    ps = [int(x) for x in spec.p]
    out, its, sts, _ = run_batch(cases, ps)
    print("statuses", {P.STATUS_NAMES[s]: sts.count(s) for s in set(sts)}, "max iterations", max(its))
    rng = np.random.default_rng(0)
    for i in rng.choice(512, 6, replace=False):
        case, p = cases[i], ps[i]
        Co, info = O.solve(case.A, p, tol=1e-12)
        Z = O.closed_form_root(case.Q, case.lam, p)
        assert O.forward_error(out[i][0], Z) <= max(1e-12, 10 * O.forward_error(Co, Z)), (i, case.n, p)
    # Every matrix satisfies the method's own accuracy floor: the coupled form from Eq. 3 keeps about
    # u kappa^(p+1) (u = 2^-53); Newton-Schulz about u kappa.
    for i, (case, p) in enumerate(zip(cases, ps)):
        Z = O.closed_form_root(case.Q, case.lam, p)
        floor = 1.1e-16 * case.kappa ** (p + 1 if p > 1 else 1) * np.sqrt(case.n)
        assert O.forward_error(out[i][0], Z) <= max(1e-10, 100 * floor), (i, case.n, p, case.kappa)


def test_batch_stats_count_every_product():
    # Per matrix of order n and k iterations: Newton-Schulz (p = 1) runs k + 1 residual products A X (full,
    # 2 n^3 flops) and k updates X T (symmetric, n^2 (n + 1)); the coupled form runs p products for M_0 and
    # p + 1 per iteration (3 for p = 3: X N, M^2, L R), all symmetric, and the verification of its stop:
    # X^p by p - 1 symmetric products, then the full product with A.
    cases, ps = make_batch(6, 64, 300, 1e3, 77)
    mats = [torch.from_numpy(c.A).to(DEV) for c in cases]
    b = P.pr_batch_init(mats, ps, P.pr_default_options(), torch.cuda.current_stream(DEV).cuda_stream)
    try:
        P.pr_batch_set_timing(b, True)
        its, _ = P.pr_batch_solve(b, len(cases), P.PR_EMU64, 1e-12)
        st = P.pr_batch_stats(b)
    finally:
        P.pr_batch_destroy(b)
    products, flops = 0, 0.0
    for c, p, k in zip(cases, ps, its):
        n = float(c.n)
        sym, full = n * n * (n + 1), 2 * n ** 3
        if p == 1:
            products += 2 * k + 1
            flops += (k + 1) * full + k * sym
        else:
            per = 3 if p == 3 else p + 1
            products += p + k * per + p
            flops += (p + k * per + p - 1) * sym + full
    assert st["products"] == products
    assert st["product_flops"] == pytest.approx(flops, rel=1e-12)
    assert st["stages_timed"] == st["stages"] and st["stage_flops_timed"] == st["product_flops"]
    assert st["stage_ms"] > 0 and st["emu_slices"] == 8 and st["launches"] > st["stages"]


def test_batch_tile_tuner_and_narrow_tiles():
    # Default options: pr_batch_init times the batch's symmetric product with 128 x 96 and 128 x 48 tiles and
    # keeps the faster; the choice is reported. Every result meets the oracle bar whichever width runs, and a
    # batch fixed at 48 gives the same products as one fixed at 96 (exact digit-pair sums): results equal
    # bit for bit wherever the two made the same stop decisions.
    cases, ps = make_batch(8, 20, 400, 1e3, 61)
    mats = [torch.from_numpy(c.A).to(DEV) for c in cases]
    b = P.pr_batch_init(mats, ps, P.pr_default_options(), torch.cuda.current_stream(DEV).cuda_stream)
    try:
        st = P.pr_batch_stats(b)
        assert st["tile_n"] in (96, 48) and st["tune_ms"] > 0
        its, sts = P.pr_batch_solve(b, len(cases), P.PR_EMU64, 1e-12)
        for i, (case, p) in enumerate(zip(cases, ps)):
            C = np.empty((case.n, case.n))
            P.pr_batch_result(b, i, C)
            Co, _ = O.solve(case.A, p, tol=1e-12)
            Z = O.closed_form_root(case.Q, case.lam, p)
            assert O.forward_error(C, Z) <= max(1e-12, 10 * O.forward_error(Co, Z)), (i, case.n, p)
    finally:
        P.pr_batch_destroy(b)
    out48, its48, _, _ = run_batch(cases, ps, tile=48)
    out96, its96, _, _ = run_batch(cases, ps, tile=96)
    for i in range(len(cases)):
        if its48[i] == its96[i]:
            assert np.array_equal(out48[i][0], out96[i][0]), i
