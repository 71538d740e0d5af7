"""pr_norms_noalloc: the norms of the initial guess for callers that cannot allocate device memory.

Some callers must not call cudaMalloc or cudaFree at all: code that runs while a CUDA graph is being
captured, latency-critical paths that cannot take the synchronisation cudaFree implies, or programs whose
device memory is already reserved by their own allocator. For them the library offers this entry point,
whose scratch is a fixed array in device memory. This test calls it through the C ABI twice in a row, with
different matrices (the second smaller, so stale scratch contents from the first call would show), and
compares each result with the norms the regular entry point (pr_init, reported by pr_stats) computes and
with the definitions (largest absolute column and row sums) evaluated on the host. A third call with a NaN
entry checks that a non-finite input shows in the result instead of being dropped by the maximum.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1703_02283_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1703_02283_gb300 import pthroot as P  # noqa: E402

DEV = torch.device("cuda:0")


def regular_norms(A, n, stream):
    h = P.pr_init(A, n, 2, None, stream)
    try:
        s = P.pr_stats(h)
    finally:
        P.pr_destroy(h)
    return s["norm_1"], s["norm_inf"]


def test_norms_noalloc_matches_regular_entry_point_twice():
    stream = torch.cuda.current_stream(DEV).cuda_stream
    for n, seed in ((700, 21), (133, 22)):
        Ah = W.spd_from_spectrum(n, 1e-2, seed).A
        A = torch.from_numpy(Ah).to(DEV)
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=DEV)
        st = P._lib.pr_norms_noalloc(ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream))
        assert st == P.PR_OK, P.pr_last_error(None)
        torch.cuda.synchronize(DEV)
        got = out.cpu().numpy()
        want = np.array(regular_norms(A, n, stream))
        np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)
        defn = np.array([np.abs(Ah).sum(axis=0).max(), np.abs(Ah).sum(axis=1).max()])
        np.testing.assert_allclose(got, defn, rtol=1e-13, atol=0)


def test_norms_noalloc_shows_a_nan_input():
    stream = torch.cuda.current_stream(DEV).cuda_stream
    Ah = W.spd_from_spectrum(90, 1e-2, 23).A.copy()
    Ah[17, 40] = np.nan
    A = torch.from_numpy(Ah).to(DEV)
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    st = P._lib.pr_norms_noalloc(ctypes.c_void_p(A.data_ptr()), 90, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream))
    assert st == P.PR_OK
    torch.cuda.synchronize(DEV)
    assert np.isnan(out.cpu().numpy()).all()


def test_norms_noalloc_rejects_sizes_beyond_the_maximum():
    A = torch.zeros((1, 1), dtype=torch.float64, device=DEV)
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    st = P._lib.pr_norms_noalloc(ctypes.c_void_p(A.data_ptr()), 65537, ctypes.c_void_p(out.data_ptr()), None)
    assert st == P.PR_EINVAL and "65536" in P.pr_last_error(None)
