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


_FRESH = r"""
import ctypes, math, sys
import torch
sys.path.insert(0, sys.argv[1])
import paper_2503_20907_gb300 as sp
from paper_2503_20907_gb300 import _lib as L
lib = sp.load(build_if_stale=False)
f = lib.spline_project_fwd_noalloc
f.restype = ctypes.c_int
f.argtypes = [ctypes.POINTER(L.SpGrid), ctypes.c_void_p, ctypes.POINTER(L.SpLines), ctypes.c_void_p, ctypes.c_void_p]
dev = torch.device("cuda")
grid = sp.Grid(64, 64, 3)
lines = sp.Lines.fan(torch.linspace(0, 2 * math.pi, 121, device=dev)[:-1].contiguous(), 130.0, 65.0, 96, -47.5, 1.0)
coef = torch.rand(64, 64, device=dev)
out = torch.empty(lines.m, device=dev)
g, Lc = grid.c(), lines.c()
stream = torch.cuda.current_stream().cuda_stream
# the first call on the device loads the array (and the kernels) under lazy module loading
assert f(ctypes.byref(g), coef.data_ptr(), ctypes.byref(Lc), out.data_ptr(), stream) == 0, lib.sp_last_error()
torch.cuda.synchronize()
free0, _ = torch.cuda.mem_get_info()
for _ in range(3):
    assert f(ctypes.byref(g), coef.data_ptr(), ctypes.byref(Lc), out.data_ptr(), stream) == 0, lib.sp_last_error()
torch.cuda.synchronize()
free1, _ = torch.cuda.mem_get_info()
print(free0, free1)
assert free0 == free1, (free0, free1)
"""


def test_noalloc_forward_takes_no_device_memory_after_its_first_call():
    """In a fresh process (no workspace left by earlier tests): after the first
    call, further calls leave the device's free memory exactly as it was."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sp.load()   # build if needed before the child loads the library as it is
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
