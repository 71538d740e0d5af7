"""The paper's custom-precision experiment on the GPU (Sec. 4.2-4.3, Fig. 2), through the C ABI.

Arithmetic mode (every operation rounded to m stored mantissa bits) is compared with the oracle's
quantized_iterates iterate by iterate, bit for bit: both sides sum every product in the order
k = 0, 1, ..., n - 1 and round every product, partial sum and update operation to nearest even from the
FP64 result, so nothing is left to rounding order. (C_0 comes from FP64 norms whose last bits may differ
between the two; at these widths its m-bit rounding does not see them.) Storage mode computes in FP64 and
rounds the input and each stored iterate: the GPU's FP64 products sum in another order than numpy's, so
iterates agree to within one unit of the m-bit grid.
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


def overlap(n, seed):
    return W.overlap_matrix(W.overlap_points(n, 20.0 * (n / 2048) ** (1 / 3), seed))


def gpu_iterates(S, p, m, mode, iterations):
    n = S.shape[0]
    o = P.pr_default_options()
    o.form = P.PR_FORM_LITERAL
    o.quant_bits = m
    o.quant_mode = mode
    o.stag_below = 0.0  # no stagnation exit: exactly the requested number of updates
    o.verify = 0
    A = torch.from_numpy(S).to(DEV)
    h = P.pr_init(A, n, p, o, torch.cuda.current_stream(DEV).cuda_stream)
    out = []
    try:
        C = torch.empty_like(A)
        P.pr_result(h, C)
        out.append(C.cpu().numpy())
        for _ in range(iterations):
            P.pr_iterate(h, 1, P.PR_FP64, 0.0)
            P.pr_result(h, C)
            out.append(C.cpu().numpy())
    finally:
        P.pr_destroy(h)
    return out


@pytest.mark.parametrize("n", [37, 64, 90])
@pytest.mark.parametrize("m,p", [(10, 2), (16, 2), (8, 1), (20, 3)])
def test_arithmetic_mode_bit_exact(n, m, p):
    S = overlap(n, 11 + n)
    want = O.quantized_iterates(S, p, m, "arithmetic", 6)
    got = gpu_iterates(S, p, m, P.PR_QUANT_ARITH, 6)
    for k in range(7):
        assert np.array_equal(got[k], want[k]), (k, float(np.max(np.abs(got[k] - want[k]))))


@pytest.mark.parametrize("m", [2, 4, 10, 23])
def test_storage_mode_within_one_grid_step(m):
    S = overlap(80, 5)
    want = O.quantized_iterates(S, 2, m, "storage", 8)
    got = gpu_iterates(S, 2, m, P.PR_QUANT_STORAGE, 8)
    for k in range(9):
        grid = np.ldexp(1.0, np.frexp(np.abs(want[k]))[1] - m - 1)  # spacing of the m-bit numbers at each value
        assert np.all(np.abs(got[k] - want[k]) <= grid + 1e-300), k
    # Every stored value lies on the m-bit grid.
    np.testing.assert_array_equal(got[-1], O.round_mantissa(got[-1], m))


def test_experiment_options_are_checked():
    S = overlap(30, 1)
    A = torch.from_numpy(S).to(DEV)
    o = P.pr_default_options()
    o.quant_bits = 10  # not the literal form
    with pytest.raises(P.PthrootError) as e:
        P.pr_init(A, 30, 2, o, torch.cuda.current_stream(DEV).cuda_stream)
    assert e.value.status == P.PR_EUNSUPPORTED
    o.form = P.PR_FORM_LITERAL
    o.quant_bits = 60
    with pytest.raises(P.PthrootError) as e:
        P.pr_init(A, 30, 2, o, torch.cuda.current_stream(DEV).cuda_stream)
    assert e.value.status == P.PR_EINVAL
