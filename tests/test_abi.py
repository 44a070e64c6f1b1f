"""The C ABI without a GPU: the library builds, loads, exports every function
that include/*.h declares, and rejects bad arguments on the host before any
CUDA call."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    sp = pytest.importorskip("paper_2503_20907_gb300")
    return sp.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("spline_project_fwd", "spline_project_adj", "spline_lines_expand", "spline_visited",
              "spline_footprint_eval", "sp_last_error", "sp_release_workspace", "sp_lines_count"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_side_argument_checks(lib):
    from paper_2503_20907_gb300 import _lib as L
    g = L.SpGrid(8, 8, 7, 0, 1.0, 0.0, 0.0)           # degree out of range
    lines = L.SpLines()
    lines.kind = L.KIND_THETA_Y
    lines.m = 4
    lines.theta = 1
    lines.y = 1
    st = lib.spline_project_fwd(ctypes.byref(g), 1, ctypes.byref(lines), 1, None)
    assert st == L.SP_EINVAL
    assert b"degree" in lib.sp_last_error()
    g = L.SpGrid(8, 8, 3, 0, -1.0, 0.0, 0.0)          # negative spacing
    assert lib.spline_project_adj(ctypes.byref(g), 1, ctypes.byref(lines), 1, None) == L.SP_EINVAL
    g = L.SpGrid(8, 8, 3, 0, 1.0, 0.0, 0.0)
    bad = L.SpLines()
    bad.kind = 7                                       # unknown kind
    assert lib.spline_project_fwd(ctypes.byref(g), 1, ctypes.byref(bad), 1, None) == L.SP_EINVAL
    assert lib.sp_lines_count(ctypes.byref(bad)) == -1
    fan = L.SpLines()
    fan.kind = L.KIND_FAN
    fan.n_view, fan.n_det, fan.view = 3, 5, 1
    fan.dso, fan.dod, fan.ddet = -1.0, 1.0, 1.0        # source distance must be > 0
    assert lib.spline_project_fwd(ctypes.byref(g), 1, ctypes.byref(fan), 1, None) == L.SP_EINVAL
    fan.dso = 10.0
    assert lib.sp_lines_count(ctypes.byref(fan)) == 15
    fan.m = 14                                         # inconsistent count
    assert lib.sp_lines_count(ctypes.byref(fan)) == -1
    g9 = L.SpGrid(1, 1, 9, 0, 1.0, 0.0, 0.0)          # degree out of range
    assert lib.spline_footprint_eval(ctypes.byref(g9), 3, 1, 1, 1, None) == L.SP_EINVAL
    gb = L.SpGrid(8, 8, 3, L.BASIS_BOX3, 1.0, 0.0, 0.0)   # the box-spline needs degree 1
    assert lib.spline_project_fwd(ctypes.byref(gb), 1, ctypes.byref(fan), 1, None) == L.SP_EINVAL
    assert b"box" in lib.sp_last_error()
    gu = L.SpGrid(8, 8, 1, 5, 1.0, 0.0, 0.0)          # unknown basis
    assert lib.spline_project_fwd(ctypes.byref(gu), 1, ctypes.byref(fan), 1, None) == L.SP_EINVAL
    assert lib.sp_version() >= 100
    t = ctypes.c_double(0.0)
    assert lib.sp_fp32_peak(2, ctypes.byref(t), None, None) == L.SP_EINVAL   # packed must be 0 or 1
    assert lib.sp_fp32_peak(0, None, None, None) == L.SP_EINVAL


def test_plan_and_batch_host_side_checks(lib):
    from paper_2503_20907_gb300 import _lib as L
    # NULL handles and bad counts are rejected before any CUDA call
    assert lib.spline_batch_count(None) == -1
    assert lib.spline_batch_queued(None, 0) == -1 and lib.spline_batch_queued(None, 1) == -1
    h = ctypes.c_void_p()
    assert lib.spline_batch_create(0, None, None, ctypes.byref(h)) == L.SP_EINVAL
    assert lib.spline_batch_fwd(None, None, None, None) == L.SP_EINVAL
    assert lib.spline_batch_adj(None, None, None, None) == L.SP_EINVAL
    assert lib.spline_batch_autotune(None, None, None, None, None) == L.SP_EINVAL
    assert lib.spline_batch_destroy(None) == L.SP_OK
    assert lib.spline_plan_set_paths(None, 0, 0) == L.SP_EINVAL


def test_conv_host_side_argument_checks(lib):
    # every case returns SP_EINVAL before any CUDA call (the pointers are
    # never dereferenced): sizes, dilation, channel pairs, NULL and
    # misaligned pointers of the tensor-core layers
    from paper_2503_20907_gb300 import _lib as L
    P = 4096                                             # a 16-byte aligned dummy address
    for args in [(0, 4, 4, 32, 32, 1), (1, 0, 4, 32, 32, 1), (1, 4, 4, 32, 32, 0), (1, 4, 4, 32, 32, 17),
                 (1, 4, 4, 16, 32, 1), (1, 4, 4, 32, 8, 1), (1, 4, 4, 1, 1, 1)]:
        assert lib.sp_conv3x3_fwd(*args, P, P, None, 0, P, None) == L.SP_EINVAL, args
        assert lib.sp_conv3x3_bwd_data(*args, P, P, None, P, None) == L.SP_EINVAL, args
        assert lib.sp_conv3x3_bwd_weight(*args, P, P, P, P, None) == L.SP_EINVAL, args
    ok = (2, 4, 4, 32, 32, 1)
    assert lib.sp_conv3x3_fwd(*ok, None, P, None, 0, P, None) == L.SP_EINVAL
    assert b"NULL" in lib.sp_last_error()
    assert lib.sp_conv3x3_fwd(*ok, P + 8, P, None, 0, P, None) == L.SP_EINVAL
    assert b"aligned" in lib.sp_last_error()
    assert lib.sp_conv3x3_bwd_data(*ok, P + 4, P, None, P, None) == L.SP_EINVAL
    assert b"aligned" in lib.sp_last_error()
    assert lib.sp_conv3x3_bwd_data(*ok, P, P, P + 2, P, None) == L.SP_EINVAL     # gate
    assert b"aligned" in lib.sp_last_error()
    assert lib.sp_conv3x3_bwd_weight(*ok, P + 2, P, P, P, None) == L.SP_EINVAL
    assert b"aligned" in lib.sp_last_error()
    assert lib.sp_conv3x3_bwd_weight(*ok, P, P + 8, P, P, None) == L.SP_EINVAL
    assert lib.sp_conv3x3_bwd_weight(*ok, P, P, None, P, None) == L.SP_EINVAL
    assert lib.sp_conv3x3_flip_weights(0, 32, P, P, None) == L.SP_EINVAL
    assert lib.sp_conv3x3_flip_weights(32, 32, None, P, None) == L.SP_EINVAL
