"""spline_project_fwd_noalloc: the forward projection for callers that cannot
let the library allocate device memory (a caller-owned memory pool, or a
pipeline that cannot take the synchronisation of cudaMalloc/cudaFree).  Its
scratch is a fixed array in the library's device memory.

It must give what spline_project_fwd gives, call after call (the array keeps
the previous call's contents), and refuse line lists that do not fit.  This
file is collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")
from paper_2503_20907_gb300 import _lib as L  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _noalloc(lib):
    f = lib.spline_project_fwd_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(L.SpGrid), ctypes.c_void_p, ctypes.POINTER(L.SpLines), ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def _rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / b.norm())


def test_noalloc_forward_matches_allocating_forward_on_consecutive_calls():
    lib = sp.load()
    f = _noalloc(lib)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        # 96 x 96 cubic fan: 180 x 144 = 25,920 lines with their own tables (~35 MB)
        (sp.Grid(96, 96, 3), sp.Lines.fan(torch.linspace(0, 2 * math.pi, 181, device=dev)[:-1].contiguous(),
                                          190.0, 95.0, 144, -71.5, 1.0), 11),
        # 80 x 64 linear parallel beam, per-view tables
        (sp.Grid(80, 64, 1, 0.8), sp.Lines.parallel(torch.linspace(0, math.pi, 121, device=dev)[:-1].contiguous(),
                                                    110, -54.5, 0.9), 12),
    ]
    for grid, lines, seed in cases:
        coef_np = workloads.ellipse_phantom(grid.nx, 12, seed, radius=0.3 * grid.nx, axes=(2.0, 0.25 * grid.nx))
        coef = torch.from_numpy(np.ascontiguousarray(coef_np[:grid.ny, :grid.nx])).to(dev)
        out = torch.full((lines.m,), float("nan"), device=dev)
        g, Lc = grid.c(), lines.c()
        st = f(ctypes.byref(g), coef.data_ptr(), ctypes.byref(Lc), out.data_ptr(), stream)
        assert st == L.SP_OK, lib.sp_last_error()
        ref = sp.spline_project_fwd(grid, coef, lines)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < TOL


def test_noalloc_forward_refuses_lists_beyond_its_scratch():
    lib = sp.load()
    f = _noalloc(lib)
    dev = torch.device("cuda")
    n = 200_000   # 200k lines with their own tables need ~275 MB
    th = torch.zeros(n, device=dev)
    yy = torch.zeros(n, device=dev)
    lines = sp.Lines.theta_y(th, yy)
    grid = sp.Grid(64, 64, 3)
    coef = torch.zeros(64, 64, device=dev)
    out = torch.zeros(n, device=dev)
    g, Lc = grid.c(), lines.c()
    st = f(ctypes.byref(g), coef.data_ptr(), ctypes.byref(Lc), out.data_ptr(), None)
    assert st == L.SP_EINVAL
    assert b"scratch" in lib.sp_last_error()
