"""Checkpoint and resume of an iteration through the C ABI (pr_export_state / pr_import_state).

A state exported part-way and imported into a fresh handle of the same matrix must continue to the same
result, bit for bit, as the handle that never stopped: in the coupled form, in Newton-Schulz, and across
the BF16 -> EMU64 ladder. A state of another matrix, or a damaged buffer, is refused; a state whose iterate
was corrupted (NaN) is caught by the stop rule on the next residual.
"""
import numpy as np
import pytest

from paper_1703_02283_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1703_02283_gb300 import pthroot as P  # noqa: E402

DEV = torch.device("cuda:0")


def stream():
    return torch.cuda.current_stream(DEV).cuda_stream


def new_handle(case, p):
    return P.pr_init(torch.from_numpy(case.A).to(DEV), case.n, p, P.pr_default_options(), stream())


def finish(h, n, bulk, bulk_steps, final):
    st, steps = P.pr_solve(h, bulk, bulk_steps, final, 1e-12)
    C = torch.empty((n, n), dtype=torch.float64, device=DEV)
    P.pr_result(h, C)
    return st, C.cpu().numpy(), P.pr_history(h), P.pr_stats(h)


@pytest.mark.parametrize("p,prec,first", [(2, P.PR_EMU64, 6), (3, P.PR_FP64, 9), (1, P.PR_EMU64, 4),
                                          (1, P.PR_BF16, 3)])
def test_resume_is_bit_identical(p, prec, first):
    case = W.spd_from_spectrum(200, 1e-2, 70 + p)
    h1, h2 = new_handle(case, p), new_handle(case, p)
    try:
        P.pr_iterate(h1, first, prec, 1e-12)
        state = P.pr_export_state(h1)
        hd = P.pr_state_header_of(state)
        assert hd.magic == 0x5052535441544531 and hd.iterations == first and hd.hist_len >= first
        # With a BF16 start the ladder continues in BF16 and then switches to EMU64.
        bulk, final = (P.PR_BF16, P.PR_EMU64) if prec == P.PR_BF16 else (prec, prec)
        st1, C1, H1, S1 = finish(h1, case.n, bulk, 100 if prec == P.PR_BF16 else 0, final)
        P.pr_import_state(h2, state)
        st2, C2, H2, S2 = finish(h2, case.n, bulk, 100 if prec == P.PR_BF16 else 0, final)
    finally:
        P.pr_destroy(h1)
        P.pr_destroy(h2)
    assert st1 == st2 and np.array_equal(C1, C2) and H1 == H2
    assert S1["iterations"] == S2["iterations"] and S1["iterations_by_precision"] == S2["iterations_by_precision"]
    assert S1["switch_iteration"] == S2["switch_iteration"]


def test_import_refuses_other_matrices_and_damaged_buffers():
    a = W.spd_from_spectrum(120, 1e-2, 80)
    b = W.spd_from_spectrum(120, 1e-2, 81)
    ha, hb, hp = new_handle(a, 2), new_handle(b, 2), new_handle(a, 3)
    try:
        P.pr_iterate(ha, 3, P.PR_EMU64, 1e-12)
        state = P.pr_export_state(ha)
        for h in (hb, hp):  # another matrix (its norms differ), another root
            with pytest.raises(P.PthrootError) as e:
                P.pr_import_state(h, state)
            assert e.value.status == P.PR_EINVAL
        bad = state.copy()
        bad[0] ^= 0xFF  # magic
        with pytest.raises(P.PthrootError) as e:
            P.pr_import_state(ha, bad)
        assert e.value.status == P.PR_EINVAL
        with pytest.raises(P.PthrootError) as e:
            P.pr_import_state(ha, state[: len(state) // 2])
        assert e.value.status == P.PR_EINVAL
    finally:
        for h in (ha, hb, hp):
            P.pr_destroy(h)


def test_corrupted_iterate_is_caught_by_the_stop_rule():
    # Fault injection on the host: a NaN written into the exported iterate X. The residual of the next
    # update is not finite and the handle stops with PR_EDIVERGED; nothing faults on the device.
    case = W.spd_from_spectrum(150, 1e-2, 90)
    h = new_handle(case, 1)
    try:
        P.pr_iterate(h, 2, P.PR_EMU64, 1e-12)
        state = P.pr_export_state(h)
        hd = P.pr_state_header_of(state)
        off = (P.ctypes.sizeof(P.pr_state_header) + 8 * hd.hist_len + (4 * hd.hist_len + 7) // 8 * 8)
        X = state[off: off + 8 * 150 * 150].view(np.float64)
        X[150 * 7 + 3] = np.nan
        P.pr_import_state(h, state)
        with pytest.raises(P.PthrootError) as e:
            P.pr_iterate(h, 10, P.PR_EMU64, 1e-12)
        assert e.value.status == P.PR_EDIVERGED
        assert not np.isfinite(P.pr_history(h)[-1])
    finally:
        P.pr_destroy(h)
