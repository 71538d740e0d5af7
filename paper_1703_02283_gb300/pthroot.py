"""Thin ctypes binding of the C ABI in include/pthroot.h (argument marshalling only).

Every function here has the name of the C entry point it calls and adds nothing to it. Matrix
arguments may be torch tensors (device or host; their ``data_ptr()`` is passed), numpy arrays (host)
or raw integer addresses. All compute happens in the library's CUDA kernels; if the shared library
is missing, importing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpthroot.so")

# enums (values fixed by include/pthroot.h)
PR_OK, PR_EINVAL, PR_ENOTSPD, PR_ENOMEM, PR_ECUDA, PR_EDIVERGED, PR_ESTAGNATED = 0, 1, 2, 3, 4, 5, 6
PR_EMAXITER, PR_ETIMEOUT, PR_EGATE, PR_ESTATE, PR_EUNSUPPORTED, PR_EINACCURATE = 7, 8, 9, 10, 11, 12
STATUS_NAMES = {0: "PR_OK", 1: "PR_EINVAL", 2: "PR_ENOTSPD", 3: "PR_ENOMEM", 4: "PR_ECUDA",
                5: "PR_EDIVERGED", 6: "PR_ESTAGNATED", 7: "PR_EMAXITER", 8: "PR_ETIMEOUT",
                9: "PR_EGATE", 10: "PR_ESTATE", 11: "PR_EUNSUPPORTED", 12: "PR_EINACCURATE"}
PR_FP64, PR_EMU64, PR_FP32X, PR_BF16, PR_FP8 = 0, 1, 2, 3, 4
PR_NPREC = 5
PREC_NAMES = {PR_FP64: "fp64", PR_EMU64: "emu64", PR_FP32X: "fp32x", PR_BF16: "bf16", PR_FP8: "fp8"}
PR_FORM_AUTO, PR_FORM_COUPLED, PR_FORM_NS, PR_FORM_LITERAL = 0, 1, 2, 3
PR_C0_EQ3, PR_C0_SCALED_I, PR_C0_POLY = 0, 1, 2
PR_QUANT_STORAGE, PR_QUANT_ARITH = 1, 2
PR_MLP_PARAMS = 4996
PR_REFINE_MAX_STEPS = 16


class pr_options(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("c0", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("stag_below", ctypes.c_double), ("stag_ratio", ctypes.c_double),
                ("sym_tol", ctypes.c_double), ("reanchor", ctypes.c_int), ("emu_slices", ctypes.c_int),
                ("stag_below_lowp", ctypes.c_double), ("c0_coef", ctypes.c_double * 4), ("gate_max", ctypes.c_double),
                ("gate_iters", ctypes.c_int), ("verify", ctypes.c_int), ("gate_fallback", ctypes.c_int),
                ("emu_tile", ctypes.c_int), ("quant_bits", ctypes.c_int), ("quant_mode", ctypes.c_int),
                ("block_sparse", ctypes.c_int)]


class pr_stats_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int), ("form", ctypes.c_int), ("c0", ctypes.c_int),
                ("iterations", ctypes.c_int), ("iterations_by_precision", ctypes.c_int * PR_NPREC),
                ("switch_iteration", ctypes.c_int), ("last_precision", ctypes.c_int),
                ("last_stop", ctypes.c_int), ("norm_1", ctypes.c_double), ("norm_inf", ctypes.c_double),
                ("last_residual", ctypes.c_double), ("gemms", ctypes.c_int64), ("gemm_flops", ctypes.c_double),
                ("launches", ctypes.c_int64), ("gemms_timed", ctypes.c_int64), ("gemm_ms", ctypes.c_double),
                ("gemm_flops_timed", ctypes.c_double), ("emu_slices", ctypes.c_int),
                ("gemms_timed_by_precision", ctypes.c_int64 * PR_NPREC),
                ("gemm_ms_by_precision", ctypes.c_double * PR_NPREC),
                ("gemm_flops_by_precision", ctypes.c_double * PR_NPREC), ("c0_gate", ctypes.c_double),
                ("true_residual", ctypes.c_double), ("prescale_log2", ctypes.c_int),
                ("emu_tile_n", ctypes.c_int * 2), ("emu_tile_split", ctypes.c_int * 2),
                ("emu_tune_ms", ctypes.c_double), ("emu_variant_ms", (ctypes.c_double * 4) * 2),
                ("ladder_restores", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("refine_cg_iterations", ctypes.c_int64), ("refine_len", ctypes.c_int),
                ("refine_residuals", ctypes.c_double * (PR_REFINE_MAX_STEPS + 1)),
                ("refine_cg", ctypes.c_int * PR_REFINE_MAX_STEPS), ("sparse_keep", ctypes.c_double),
                ("sparse_products", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["emu_variant_ms"] = [list(r) for r in self.emu_variant_ms]
        for k in ("iterations_by_precision", "gemms_timed_by_precision", "gemm_ms_by_precision",
                  "gemm_flops_by_precision", "emu_tile_n", "emu_tile_split"):
            d[k] = list(getattr(self, k))
        d["refine_residuals"] = list(self.refine_residuals)[: self.refine_len]
        d["refine_cg"] = list(self.refine_cg)[: max(self.refine_len - 1, 0)]
        return d


class pr_state_header(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint64), ("n", ctypes.c_int64), ("version", ctypes.c_int32),
                ("p", ctypes.c_int32), ("form", ctypes.c_int32), ("c0", ctypes.c_int32),
                ("norm_1", ctypes.c_double), ("norm_inf", ctypes.c_double), ("state_ready", ctypes.c_int32),
                ("state_level", ctypes.c_int32), ("lp_stale", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("iterations_by_precision", ctypes.c_int32 * PR_NPREC), ("switch_iteration", ctypes.c_int32),
                ("last_precision", ctypes.c_int32), ("hist_len", ctypes.c_int32), ("n_mats", ctypes.c_int32),
                ("ldl", ctypes.c_int32), ("reserved", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("last_residual", ctypes.c_double)]


class pr_batch_matrix_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int), ("form", ctypes.c_int), ("status", ctypes.c_int),
                ("iterations", ctypes.c_int), ("norm_1", ctypes.c_double), ("norm_inf", ctypes.c_double),
                ("prescale_log2", ctypes.c_int), ("true_residual", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class pr_batch_stats_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("stages", ctypes.c_int64), ("products", ctypes.c_int64),
                ("product_flops", ctypes.c_double), ("stages_timed", ctypes.c_int64), ("stage_ms", ctypes.c_double),
                ("stage_flops_timed", ctypes.c_double), ("emu_slices", ctypes.c_int), ("tile_n", ctypes.c_int),
                ("tune_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_handle_t = ctypes.c_void_p
_dptr = ctypes.c_void_p


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1703_02283_gb300.build` "
                          "(the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "pr_version": (ctypes.c_int, []),
        "pr_default_options": (None, [ctypes.POINTER(pr_options)]),
        "pr_init": (ctypes.c_int, [ctypes.POINTER(_handle_t), _dptr, ctypes.c_int64, ctypes.c_int,
                                   ctypes.POINTER(pr_options), ctypes.c_void_p]),
        "pr_load": (ctypes.c_int, [_handle_t, _dptr]),
        "pr_set_timing": (ctypes.c_int, [_handle_t, ctypes.c_int]),
        "pr_iterate": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_int)]),
        "pr_solve": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_int)]),
        "pr_solve_ladder": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
        "pr_residual": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "pr_refine": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
        "pr_set_iterate": (ctypes.c_int, [_handle_t, _dptr]),
        "pr_result": (ctypes.c_int, [_handle_t, _dptr]),
        "pr_stop_rule": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(pr_options)]),
        "pr_batch_init": (ctypes.c_int, [ctypes.POINTER(_handle_t), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(pr_options), ctypes.c_void_p]),
        "pr_batch_load": (ctypes.c_int, [_handle_t, ctypes.POINTER(ctypes.c_void_p)]),
        "pr_batch_solve": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
        "pr_batch_result": (ctypes.c_int, [_handle_t, ctypes.c_int, _dptr]),
        "pr_batch_history": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
        "pr_batch_launches": (ctypes.c_int64, [_handle_t]),
        "pr_batch_matrix": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.POINTER(pr_batch_matrix_t)]),
        "pr_batch_stats": (ctypes.c_int, [_handle_t, ctypes.POINTER(pr_batch_stats_t)]),
        "pr_batch_set_timing": (ctypes.c_int, [_handle_t, ctypes.c_int]),
        "pr_batch_last_error": (ctypes.c_char_p, [_handle_t]),
        "pr_batch_destroy": (ctypes.c_int, [_handle_t]),
        "pr_features": (ctypes.c_int, [_handle_t, ctypes.POINTER(ctypes.c_double)]),
        "pr_spectral_bounds": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]),
        "pr_set_initial_guess": (ctypes.c_int, [_handle_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "pr_mlp_create": (ctypes.c_int, [ctypes.POINTER(_handle_t), _dptr, ctypes.c_int, ctypes.c_void_p]),
        "pr_mlp_forward": (ctypes.c_int, [_handle_t, _dptr, ctypes.c_int, _dptr]),
        "pr_mlp_loss_grad": (ctypes.c_int, [_handle_t, _dptr, _dptr, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                            _dptr]),
        "pr_mlp_adam_step": (ctypes.c_int, [_handle_t, _dptr, _dptr, ctypes.c_int, ctypes.c_float,
                                            ctypes.POINTER(ctypes.c_float)]),
        "pr_mlp_get_params": (ctypes.c_int, [_handle_t, _dptr]),
        "pr_mlp_destroy": (ctypes.c_int, [_handle_t]),
        "pr_norms_noalloc": (ctypes.c_int, [_dptr, ctypes.c_int64, _dptr, ctypes.c_void_p]),
        "pr_matmul": (ctypes.c_int, [ctypes.c_int, _dptr, _dptr, ctypes.c_int64, ctypes.c_int, _dptr,
                                     ctypes.c_void_p]),
        "pr_matmul_emu": (ctypes.c_int, [ctypes.c_int, _dptr, _dptr, ctypes.c_int64, ctypes.c_int, _dptr,
                                     ctypes.c_void_p]),
        "pr_matmul_emu_tiled": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dptr, _dptr, ctypes.c_int64,
                                               ctypes.c_int, _dptr, ctypes.c_void_p]),
        "pr_state_size": (ctypes.c_int, [_handle_t, ctypes.POINTER(ctypes.c_size_t)]),
        "pr_export_state": (ctypes.c_int, [_handle_t, ctypes.c_void_p, ctypes.c_size_t]),
        "pr_import_state": (ctypes.c_int, [_handle_t, ctypes.c_void_p, ctypes.c_size_t]),
        "pr_selftest_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
        "pr_stats": (ctypes.c_int, [_handle_t, ctypes.POINTER(pr_stats_t)]),
        "pr_history": (ctypes.c_int, [_handle_t, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]),
        "pr_destroy": (ctypes.c_int, [_handle_t]),
        "pr_last_error": (ctypes.c_char_p, [_handle_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


class PthrootError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _ptr(x) -> int:
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch.Tensor
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy.ndarray
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _check(status: int, h=None, allowed=(PR_OK,)) -> int:
    if status not in allowed:
        raise PthrootError(status, (_lib.pr_last_error(h) or b"").decode())
    return status


def pr_version() -> int:
    return _lib.pr_version()


def pr_default_options() -> pr_options:
    o = pr_options()
    _lib.pr_default_options(ctypes.byref(o))
    return o


def pr_init(A, n: int, p: int, options: pr_options | None = None, stream: int = 0) -> int:
    """Returns the handle; raises PthrootError on a non-zero status."""
    h = _handle_t()
    st = _lib.pr_init(ctypes.byref(h), _ptr(A), int(n), int(p),
                      ctypes.byref(options) if options is not None else None, ctypes.c_void_p(stream))
    _check(st, None)
    return h.value


def pr_load(h: int, A) -> None:
    _check(_lib.pr_load(h, _ptr(A)), h)


def pr_set_timing(h: int, on: bool) -> None:
    _check(_lib.pr_set_timing(h, 1 if on else 0), h)


STOPS = (PR_OK, PR_ESTAGNATED, PR_EMAXITER, PR_EINACCURATE)


def pr_iterate(h: int, max_steps: int, precision: int, tol: float) -> tuple[int, int]:
    """Returns (status, steps_done); stop statuses (PR_OK, PR_ESTAGNATED, PR_EMAXITER, PR_EINACCURATE) do not
    raise."""
    d = ctypes.c_int(0)
    st = _lib.pr_iterate(h, int(max_steps), int(precision), float(tol), ctypes.byref(d))
    _check(st, h, STOPS)
    return st, d.value


def pr_solve(h: int, bulk_precision: int, bulk_steps: int, final_precision: int, tol: float) -> tuple[int, int]:
    d = ctypes.c_int(0)
    st = _lib.pr_solve(h, int(bulk_precision), int(bulk_steps), int(final_precision), float(tol), ctypes.byref(d))
    _check(st, h, STOPS)
    return st, d.value


def pr_solve_ladder(h: int, precisions, max_steps, tol: float) -> tuple[int, int]:
    """precisions: the rungs in order; max_steps: per-rung update limits (None: none). Returns (status, steps)."""
    k = len(precisions)
    pr_ = (ctypes.c_int * k)(*[int(x) for x in precisions])
    ms = None if max_steps is None else (ctypes.c_int * k)(*[int(x) for x in max_steps])
    d = ctypes.c_int(0)
    st = _lib.pr_solve_ladder(h, k, pr_, ms, float(tol), ctypes.byref(d))
    _check(st, h, STOPS)
    return st, d.value


def pr_residual(h: int, precision: int = PR_FP64) -> float:
    r = ctypes.c_double(0.0)
    _check(_lib.pr_residual(h, int(precision), ctypes.byref(r)), h)
    return r.value


def pr_refine(h: int, precision: int, inner_precision: int, max_steps: int, tol: float, cg_max: int,
              cg_tol: float) -> tuple[int, int]:
    """Returns (status, corrections kept); stop statuses (PR_OK, PR_ESTAGNATED, PR_EMAXITER, PR_EINACCURATE) do
    not raise."""
    d = ctypes.c_int(0)
    st = _lib.pr_refine(h, int(precision), int(inner_precision), int(max_steps), float(tol), int(cg_max),
                        float(cg_tol), ctypes.byref(d))
    _check(st, h, STOPS)
    return st, d.value


def pr_set_iterate(h: int, X) -> None:
    _check(_lib.pr_set_iterate(h, _ptr(X)), h)


def pr_result(h: int, C_out) -> None:
    _check(_lib.pr_result(h, _ptr(C_out)), h)


def pr_stop_rule(hist, prec, tol: float, options: pr_options | None = None) -> int:
    n = len(hist)
    h = (ctypes.c_double * max(n, 1))(*hist)
    q = (ctypes.c_int * max(n, 1))(*prec)
    return _lib.pr_stop_rule(h, q, n, float(tol), ctypes.byref(options) if options is not None else None)


def pr_features(h: int) -> list[float]:
    out = (ctypes.c_double * 8)()
    _check(_lib.pr_features(h, out), h)
    return list(out)


def pr_spectral_bounds(h: int, iters: int = 60) -> tuple[float, float]:
    """(lambda_min estimate from the current iterate, lambda_max estimate) of the loaded A."""
    lo, hi = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib.pr_spectral_bounds(h, int(iters), ctypes.byref(lo), ctypes.byref(hi)), h)
    return lo.value, hi.value


def pr_set_initial_guess(h: int, kind: int, coef=None) -> None:
    c = None if coef is None else (ctypes.c_double * 4)(*[float(x) for x in coef])
    _check(_lib.pr_set_initial_guess(h, int(kind), c), h)


def pr_mlp_create(params, max_batch: int, stream: int = 0) -> int:
    m = _handle_t()
    _check(_lib.pr_mlp_create(ctypes.byref(m), _ptr(params), int(max_batch), ctypes.c_void_p(stream)))
    return m.value


def pr_mlp_forward(m: int, X, B: int, Y) -> None:
    _check(_lib.pr_mlp_forward(m, _ptr(X), int(B), _ptr(Y)))


def pr_mlp_loss_grad(m: int, X, T, B: int, grad=None) -> float:
    loss = ctypes.c_float(0.0)
    _check(_lib.pr_mlp_loss_grad(m, _ptr(X), _ptr(T), int(B), ctypes.byref(loss),
                                 _ptr(grad) if grad is not None else None))
    return loss.value


def pr_mlp_adam_step(m: int, X, T, B: int, lr: float) -> float:
    loss = ctypes.c_float(0.0)
    _check(_lib.pr_mlp_adam_step(m, _ptr(X), _ptr(T), int(B), float(lr), ctypes.byref(loss)))
    return loss.value


def pr_mlp_get_params(m: int, params) -> None:
    _check(_lib.pr_mlp_get_params(m, _ptr(params)))


def pr_mlp_destroy(m: int) -> None:
    _check(_lib.pr_mlp_destroy(m))


def pr_norms_noalloc(A, n: int, out, stream: int = 0) -> None:
    _check(_lib.pr_norms_noalloc(_ptr(A), int(n), _ptr(out), ctypes.c_void_p(stream)), None)


def pr_matmul(precision: int, X, Y, n: int, sym: bool, P, stream: int = 0) -> None:
    _check(_lib.pr_matmul(int(precision), _ptr(X), _ptr(Y), int(n), 1 if sym else 0, _ptr(P),
                          ctypes.c_void_p(stream)), None)


def pr_export_state(h: int):
    """The handle's iteration state as a numpy uint8 array (layout: pr_state_header, then the payload)."""
    import numpy as np
    size = ctypes.c_size_t(0)
    _check(_lib.pr_state_size(h, ctypes.byref(size)), h)
    buf = np.zeros(size.value, dtype=np.uint8)
    _check(_lib.pr_export_state(h, buf.ctypes.data, buf.nbytes), h)
    return buf


def pr_import_state(h: int, buf) -> None:
    _check(_lib.pr_import_state(h, buf.ctypes.data, buf.nbytes), h)


def pr_state_header_of(buf) -> pr_state_header:
    return pr_state_header.from_buffer_copy(bytes(buf[:ctypes.sizeof(pr_state_header)]))


def pr_selftest_wait(stream: int = 0) -> tuple[int, float]:
    """(status, seconds waited): PR_ETIMEOUT is the expected status."""
    w = ctypes.c_double(0.0)
    st = _lib.pr_selftest_wait(ctypes.c_void_p(stream), ctypes.byref(w))
    return st, w.value


def pr_matmul_emu(slices: int, X, Y, n: int, sym: bool, P, stream: int = 0) -> None:
    _check(_lib.pr_matmul_emu(int(slices), _ptr(X), _ptr(Y), int(n), 1 if sym else 0, _ptr(P),
                              ctypes.c_void_p(stream)), None)


def pr_matmul_emu_tiled(slices: int, tile_n: int, split: int, X, Y, n: int, sym: bool, P, stream: int = 0) -> None:
    _check(_lib.pr_matmul_emu_tiled(int(slices), int(tile_n), int(split), _ptr(X), _ptr(Y), int(n), 1 if sym else 0,
                                    _ptr(P), ctypes.c_void_p(stream)), None)


def pr_stats(h: int) -> dict:
    s = pr_stats_t()
    _check(_lib.pr_stats(h, ctypes.byref(s)), h)
    return s.as_dict()


def pr_history(h: int) -> list[float]:
    ln = ctypes.c_int(0)
    _check(_lib.pr_history(h, None, 0, ctypes.byref(ln)), h)
    buf = (ctypes.c_double * max(ln.value, 1))()
    _check(_lib.pr_history(h, buf, ln.value, ctypes.byref(ln)), h)
    return list(buf[: ln.value])


def pr_destroy(h: int) -> None:
    _check(_lib.pr_destroy(h), None)


def _bcheck(status: int, b=None, allowed=(PR_OK,)) -> int:
    if status not in allowed:
        raise PthrootError(status, (_lib.pr_batch_last_error(b) or b"").decode())
    return status


def pr_batch_init(mats, ps, options: pr_options | None = None, stream: int = 0) -> int:
    """mats: sequence of square FP64 matrices (torch tensors or numpy arrays); ps: roots."""
    count = len(mats)
    n = (ctypes.c_int64 * count)(*[int(m.shape[0]) for m in mats])
    p = (ctypes.c_int * count)(*[int(x) for x in ps])
    ptrs = (ctypes.c_void_p * count)(*[_ptr(m) for m in mats])
    b = _handle_t()
    _bcheck(_lib.pr_batch_init(ctypes.byref(b), count, n, p, ptrs,
                               ctypes.byref(options) if options is not None else None, ctypes.c_void_p(stream)))
    return b.value


def pr_batch_load(b: int, mats) -> None:
    """Replaces the matrices of a batch (same orders) and restarts every solve."""
    ptrs = (ctypes.c_void_p * len(mats))(*[_ptr(m) for m in mats])
    _bcheck(_lib.pr_batch_load(b, ptrs), b)


def pr_batch_solve(b: int, count: int, precision: int, tol: float) -> tuple[list, list]:
    its = (ctypes.c_int * count)()
    sts = (ctypes.c_int * count)()
    _bcheck(_lib.pr_batch_solve(b, int(precision), float(tol), its, sts), b)
    return list(its), list(sts)


def pr_batch_result(b: int, i: int, C_out) -> None:
    _bcheck(_lib.pr_batch_result(b, int(i), _ptr(C_out)), b)


def pr_batch_history(b: int, i: int) -> list[float]:
    ln = ctypes.c_int(0)
    _bcheck(_lib.pr_batch_history(b, int(i), None, 0, ctypes.byref(ln)), b)
    buf = (ctypes.c_double * max(ln.value, 1))()
    _bcheck(_lib.pr_batch_history(b, int(i), buf, ln.value, ctypes.byref(ln)), b)
    return list(buf[: ln.value])


def pr_batch_matrix(b: int, i: int) -> dict:
    s = pr_batch_matrix_t()
    _bcheck(_lib.pr_batch_matrix(b, int(i), ctypes.byref(s)), b)
    return s.as_dict()


def pr_batch_launches(b: int) -> int:
    return int(_lib.pr_batch_launches(b))


def pr_batch_stats(b: int) -> dict:
    s = pr_batch_stats_t()
    _bcheck(_lib.pr_batch_stats(b, ctypes.byref(s)), b)
    return s.as_dict()


def pr_batch_set_timing(b: int, on: bool) -> None:
    _bcheck(_lib.pr_batch_set_timing(b, 1 if on else 0), b)


def pr_batch_destroy(b: int) -> None:
    _bcheck(_lib.pr_batch_destroy(b))


def pr_last_error(h: int | None = None) -> str:
    return (_lib.pr_last_error(h) or b"").decode()
