"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/wmc.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wmc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_00082_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declarations_are_all_exported(lib):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/wmc.h but not exported"


def test_binding_lists_every_declared_entry_point():
    from paper_1806_00082_gb300 import wmc
    assert sorted(wmc.EXPORTS) == _declared()


def test_params_struct_layout_matches_header(lib):
    from paper_1806_00082_gb300 import wmc
    assert ctypes.sizeof(wmc.Params) == 56
    assert ctypes.sizeof(wmc.Counters) == 72


def test_host_side_argument_checks(lib):
    """Argument errors return at once, before any device work."""
    from paper_1806_00082_gb300 import wmc
    import wmc_inputs as wi
    L = wmc.load()
    p = wmc.Params.of(wi.BARRIER_100)
    assert L.wmc_workspace_size(ctypes.byref(p)) > 0
    bad = wmc.Params.of(wi.BARRIER_100, Q=31)
    assert L.wmc_workspace_size(ctypes.byref(bad)) == 0
    assert L.wmc_init(ctypes.byref(bad), ctypes.c_void_p(256), 1 << 30, None) == 1
    # a drift of a cell or more per step is rejected
    fast = wmc.Params.of(wi.BARRIER_100, dt_s=1e-13)
    assert L.wmc_workspace_size(ctypes.byref(fast)) == 0
    # misaligned or short workspace
    assert L.wmc_init(ctypes.byref(p), ctypes.c_void_p(255), 1 << 30, None) == 1
    assert L.wmc_init(ctypes.byref(p), ctypes.c_void_p(256), 16, None) == 1
    # null buffers
    assert L.wmc_step(ctypes.byref(p), None, 1, None, None, None) == 1
    assert L.wmc_run(ctypes.byref(p), None, None, None, 1, 1, 0, 1, None, None) == 1
    assert L.wmc_kernel_eval(ctypes.byref(p), None, None, 0, 0, None, None, None) == 1
    assert L.wmc_check_wait(ctypes.byref(p), None, 1000, ctypes.c_void_p(256), None) == 1
    assert L.wmc_check_wait(ctypes.byref(p), ctypes.c_void_p(256), 1 << 40, ctypes.c_void_p(256), None) == 1
    assert L.wmc_step_timing_read(None) == 1
    assert L.wmc_step_timing(0) == 0
    assert L.wmc_status_string(3) == b"gamma dt >= 1"


def test_workspace_layout_scales():
    from paper_1806_00082_gb300 import wmc
    import wmc_inputs as wi
    s1 = wmc.workspace_size(wmc.Params.of(wi.BARRIER_100))
    s3 = wmc.workspace_size(wmc.Params.of(wi.DOUBLE_BARRIER_16384))
    assert 0 < s1 < s3 < 512 * 2 ** 20
