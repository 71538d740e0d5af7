"""The C-ABI library loads and exports every entry point declared in include/*.h; host-side argument
checks return their status codes before any device work (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pr_init", "pr_iterate", "pr_residual", "pr_result", "pr_destroy", "pr_solve"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1703_02283_gb300 import pthroot as P
    lib = ctypes.CDLL(P.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_host_side_argument_checks():
    from paper_1703_02283_gb300 import pthroot as P
    o = P.pr_default_options()
    assert (o.form, o.c0, o.max_iter, o.stag_below, o.stag_ratio, o.reanchor) == (0, 0, 100, 1e-3, 0.5, 1)
    assert o.stag_below_lowp == 0.5
    assert P.pr_version() >= 100
    lib = P._lib
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    assert lib.pr_init(None, dummy, 4, 2, None, None) == P.PR_EINVAL
    assert lib.pr_init(ctypes.byref(h), None, 4, 2, None, None) == P.PR_EINVAL
    assert lib.pr_init(ctypes.byref(h), dummy, 0, 2, None, None) == P.PR_EINVAL
    assert lib.pr_init(ctypes.byref(h), dummy, 4, 0, None, None) == P.PR_EINVAL
    bad = P.pr_default_options()
    bad.form = P.PR_FORM_NS
    assert lib.pr_init(ctypes.byref(h), dummy, 4, 2, ctypes.byref(bad), None) == P.PR_EINVAL
    assert "Newton-Schulz" in P.pr_last_error(None)
    o = P.pr_default_options()
    assert list(o.c0_coef) == [1.0, 0.0, 0.0, 0.0] and o.gate_max == 0.9 and o.gate_iters == 30
    bad = P.pr_default_options()
    bad.c0 = 7
    assert lib.pr_init(ctypes.byref(h), dummy, 4, 2, ctypes.byref(bad), None) == P.PR_EINVAL
    assert h.value is None
    assert lib.pr_iterate(None, 1, P.PR_FP64, 1e-12, None) == P.PR_ESTATE
    assert lib.pr_destroy(None) == P.PR_OK


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the size and field offsets the C compiler gives the header."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    from paper_1703_02283_gb300 import pthroot as P
    classes = {"pr_options": P.pr_options, "pr_stats_t": P.pr_stats_t, "pr_batch_stats_t": P.pr_batch_stats_t,
               "pr_state_header": P.pr_state_header}
    fields = {st: [f for f, _ in cls._fields_] for st, cls in classes.items()}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pthroot.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.split("\n") if line)
    for st, cls in classes.items():
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
