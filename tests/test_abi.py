"""The C-ABI library loads and exports every entry point include/dwt.h
declares; argument checks that need no GPU return their status codes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dwt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dwt\w*)\s*\(", src)))


@pytest.fixture(scope="module")
def libdwt():
    from paper_1605_00561_gb300 import build
    build.build()
    from paper_1605_00561_gb300 import dwt
    return dwt


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dwt_plan_create", "dwt_plan_set_scheme", "dwt2_forward", "dwt2_inverse",
                     "dwt_batch_submit", "dwt_plan_destroy", "dwt_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libdwt):
    lib = libdwt.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding covers every declared function under the same name
    assert set(declared_functions()) <= set(libdwt.EXPORTS)


def test_status_strings_and_version(libdwt):
    assert libdwt.dwt_version().count(".") == 2
    assert libdwt.dwt_status_string(libdwt.DWT_OK) == "ok"
    assert "invalid" in libdwt.dwt_status_string(libdwt.DWT_EINVAL)
    assert libdwt.dwt_status_string(99) == "unknown status"


def test_invalid_arguments_rejected_before_any_cuda_call(libdwt):
    lib = libdwt.lib()
    out = ctypes.c_void_p()
    assert lib.dwt_plan_create(0, 5, 0, 0, 0, ctypes.byref(out)) == libdwt.DWT_EINVAL
    assert lib.dwt_plan_create((1 << 28) + 1, 5, 0, 0, 0, ctypes.byref(out)) == libdwt.DWT_EINVAL
    assert lib.dwt_plan_create(5, 2 ** 31 - 1, 0, 0, 0, ctypes.byref(out)) == libdwt.DWT_EINVAL
    assert lib.dwt_plan_create(5, 5, 0, -1, 0, ctypes.byref(out)) == libdwt.DWT_EINVAL
    assert lib.dwt_plan_create(4, 4, 0, 3, 0, ctypes.byref(out)) == libdwt.DWT_EINVAL  # 2 halvings max
    assert lib.dwt_plan_create(4, 4, 7, 1, 0, ctypes.byref(out)) == libdwt.DWT_EINVAL
    assert lib.dwt_plan_create(4, 4, libdwt.DWT_CDF97, 1, libdwt.DWT_I32, ctypes.byref(out)) == \
        libdwt.DWT_EUNSUPPORTED
    # DD 13/7 runs in float32 only
    assert lib.dwt_plan_create(4, 4, libdwt.DWT_DD137, 1, libdwt.DWT_F16S, ctypes.byref(out)) == \
        libdwt.DWT_EUNSUPPORTED
    assert lib.dwt_plan_create(4, 4, libdwt.DWT_DD137, 1, libdwt.DWT_I32, ctypes.byref(out)) == \
        libdwt.DWT_EUNSUPPORTED
    assert lib.dwt_plan_create(4, 4, 0, 1, 0, None) == libdwt.DWT_EINVAL
    assert lib.dwt2_forward(None, None, 0, None, 0, None) == libdwt.DWT_EINVAL
    assert lib.dwt_plan_destroy(None) == libdwt.DWT_EINVAL
    assert lib.dwt_batch_submit(None, -1, None, None) == libdwt.DWT_EINVAL


def test_binding_raises_on_missing_library(monkeypatch, tmp_path):
    from paper_1605_00561_gb300 import dwt
    monkeypatch.setattr(dwt, "_lib", None)
    monkeypatch.setattr(dwt, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        dwt.lib()


def test_wait_limits_and_injection_arguments(libdwt):
    lib = libdwt.lib()
    assert lib.dwt_set_wait_limits(0, 0) == libdwt.DWT_OK
    assert lib.dwt_debug_inject(libdwt.DWT_INJECT_NONE, 0, 0) == libdwt.DWT_OK
    assert lib.dwt_debug_inject(4, 0, 1) == libdwt.DWT_EINVAL
    assert lib.dwt_debug_inject(-1, 0, 1) == libdwt.DWT_EINVAL
    assert lib.dwt_debug_inject(libdwt.DWT_INJECT_ENOMEM, -1, 1) == libdwt.DWT_EINVAL
    assert lib.dwt_debug_inject(libdwt.DWT_INJECT_ENOMEM, 0, -1) == libdwt.DWT_EINVAL
    assert lib.dwt_debug_inject(libdwt.DWT_INJECT_NONE, 0, 0) == libdwt.DWT_OK


def test_scheme_counts_reproduce_the_papers_table(libdwt, golden):
    """Multiply-accumulates per quadruple and barriers of the programs the
    kernels run (counted at compile time from their step lists) against the
    paper's Table of operations and barriers (Sec. 5): all 30 rows."""
    wl = {"CDF 5/3": libdwt.DWT_CDF53, "CDF 9/7": libdwt.DWT_CDF97, "DD 13/7": libdwt.DWT_DD137}
    rows = golden("op_barrier_counts.txt")
    assert len(rows) == 30
    for wavelet, scheme, barriers, ops in rows:
        name = scheme.lower()
        m, b, w = libdwt.dwt_scheme_counts(wl[wavelet], libdwt.SCHEMES[name])
        assert (m, b) == (int(ops), int(barriers)), (wavelet, scheme, m, b)
        assert w >= b  # each barrier step publishes at least one subband
    with pytest.raises(libdwt.DwtError):
        libdwt.dwt_scheme_counts(7, libdwt.SCHEMES["sweldens"])
