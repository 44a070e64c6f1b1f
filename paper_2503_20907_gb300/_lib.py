"""ctypes binding of libspline_project.so (C ABI in include/spline_project.h).

Argument marshalling only: every step of the projector runs in the library's
CUDA kernels.  There is no CPU or PyTorch fallback; if the library cannot be
built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import build as _build

SP_OK, SP_EINVAL, SP_ENOMEM, SP_ECUDA, SP_EUNSUPPORTED = 0, -1, -2, -3, -5
BASIS_BSPLINE, BASIS_BOX3 = 0, 1
KIND_THETA_Y, KIND_POINTS, KIND_PARALLEL, KIND_FAN = 0, 1, 2, 3

_lib = None


class SpGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("basis", ctypes.c_int32), ("h", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float)]


class SpLines(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_view", ctypes.c_int32), ("n_det", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("m", ctypes.c_int64),
                ("theta", ctypes.c_void_p), ("y", ctypes.c_void_p), ("src", ctypes.c_void_p),
                ("dst", ctypes.c_void_p), ("view", ctypes.c_void_p),
                ("det0", ctypes.c_float), ("ddet", ctypes.c_float),
                ("dso", ctypes.c_float), ("dod", ctypes.c_float)]


class SplineError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"spline_project status {status}: {msg}")
        self.status = status


EXPORTED = ("sp_lines_count", "spline_project_fwd", "spline_project_adj", "spline_lines_expand",
            "spline_footprint_eval", "spline_visited", "sp_release_workspace", "sp_last_error",
            "sp_version", "sp_fp32_peak", "spline_plan_create", "spline_plan_prepare", "spline_plan_fwd",
            "spline_plan_adj", "spline_plan_lines", "spline_plan_record_bytes", "spline_plan_set_records",
            "spline_plan_destroy",
            "spline_plan_stats",
            "spline_project_fwd_noalloc", "spline_plan_cgls", "spline_plan_set_paths",
            "spline_plan_autotune", "spline_batch_create", "spline_batch_prepare", "spline_batch_fwd",
            "spline_batch_adj", "spline_batch_autotune", "spline_batch_count", "spline_batch_queued",
            "spline_batch_destroy",
            "sp_conv3x3_fwd", "sp_conv3x3_bwd_data", "sp_conv3x3_bwd_weight", "sp_conv3x3_flip_weights")


def load(build_if_stale: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the in-tree CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_stale else _build.LIB
    if not path.exists():
        raise RuntimeError(f"CUDA library missing: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(str(path))
    P, st = ctypes.c_void_p, ctypes.c_int
    G, L = ctypes.POINTER(SpGrid), ctypes.POINTER(SpLines)
    lib.sp_lines_count.restype = ctypes.c_int64
    lib.sp_lines_count.argtypes = [L]
    for name, args in (("spline_project_fwd", [G, P, L, P, P]),
                       ("spline_project_adj", [G, P, L, P, P]),
                       ("spline_lines_expand", [L, P, P, P]),
                       ("spline_footprint_eval", [G, ctypes.c_int64, P, P, P, P]),
                       ("spline_visited", [G, L, P, P, P, P])):
        f = getattr(lib, name)
        f.restype = st
        f.argtypes = args
    lib.spline_plan_create.restype = st
    lib.spline_plan_create.argtypes = [G, L, ctypes.POINTER(ctypes.c_void_p)]
    lib.spline_plan_prepare.restype = st
    lib.spline_plan_prepare.argtypes = [P, P]
    lib.spline_plan_fwd.restype = st
    lib.spline_plan_fwd.argtypes = [P, P, P, P]
    lib.spline_plan_adj.restype = st
    lib.spline_plan_adj.argtypes = [P, P, P, P]
    lib.spline_plan_lines.restype = ctypes.c_int64
    lib.spline_plan_lines.argtypes = [P]
    lib.spline_plan_record_bytes.restype = ctypes.c_int64
    lib.spline_plan_record_bytes.argtypes = [P]
    lib.spline_plan_set_records.restype = st
    lib.spline_plan_set_records.argtypes = [P, ctypes.c_int32]
    lib.spline_plan_stats.restype = st
    lib.spline_plan_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.spline_project_fwd_noalloc.restype = st
    lib.spline_project_fwd_noalloc.argtypes = [G, P, L, P, P]
    lib.spline_plan_cgls.restype = st
    lib.spline_plan_cgls.argtypes = [P, P, P, ctypes.c_int32, P, P]
    lib.spline_plan_set_paths.restype = st
    lib.spline_plan_set_paths.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
    lib.spline_plan_autotune.restype = st
    lib.spline_plan_autotune.argtypes = [P, P, P, P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_float)]
    lib.spline_batch_create.restype = st
    lib.spline_batch_create.argtypes = [ctypes.c_int32, G, L, ctypes.POINTER(ctypes.c_void_p)]
    for name in ("spline_batch_fwd", "spline_batch_adj"):
        getattr(lib, name).restype = st
        getattr(lib, name).argtypes = [P, P, P, P]
    lib.spline_batch_prepare.restype = st
    lib.spline_batch_prepare.argtypes = [P, P]
    lib.spline_batch_autotune.restype = st
    lib.spline_batch_autotune.argtypes = [P, P, P, P, P]
    lib.spline_batch_count.restype = ctypes.c_int32
    lib.spline_batch_count.argtypes = [P]
    lib.spline_batch_queued.restype = ctypes.c_int32
    lib.spline_batch_queued.argtypes = [P, ctypes.c_int32]
    lib.spline_batch_destroy.restype = st
    lib.spline_batch_destroy.argtypes = [P]
    i32 = ctypes.c_int32
    lib.sp_conv3x3_fwd.restype = st
    lib.sp_conv3x3_fwd.argtypes = [i32, i32, i32, i32, i32, i32, P, P, P, i32, P, P]
    lib.sp_conv3x3_bwd_data.restype = st
    lib.sp_conv3x3_bwd_data.argtypes = [i32, i32, i32, i32, i32, i32, P, P, P, P, P]
    lib.sp_conv3x3_bwd_weight.restype = st
    lib.sp_conv3x3_bwd_weight.argtypes = [i32, i32, i32, i32, i32, i32, P, P, P, P, P]
    lib.sp_conv3x3_flip_weights.restype = st
    lib.sp_conv3x3_flip_weights.argtypes = [i32, i32, P, P, P]
    lib.spline_plan_destroy.restype = st
    lib.spline_plan_destroy.argtypes = [P]
    lib.sp_release_workspace.restype = st
    lib.sp_release_workspace.argtypes = []
    lib.sp_last_error.restype = ctypes.c_char_p
    lib.sp_version.restype = ctypes.c_int32
    lib.sp_fp32_peak.restype = st
    lib.sp_fp32_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), P]
    _lib = lib
    return lib


def _check(status: int):
    if status != SP_OK:
        raise SplineError(status, load().sp_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    return t.contiguous()


@dataclass
class Grid:
    """nx x ny nodes with spacing h centred at (cx, cy).  basis BASIS_BSPLINE:
    tensor-product B-splines of degree 0..3; BASIS_BOX3: the 3-direction
    box-spline (degree 1)."""
    nx: int
    ny: int
    degree: int
    h: float = 1.0
    cx: float = 0.0
    cy: float = 0.0
    basis: int = BASIS_BSPLINE

    def c(self) -> SpGrid:
        return SpGrid(int(self.nx), int(self.ny), int(self.degree), int(self.basis), float(self.h),
                      float(self.cx), float(self.cy))


class Lines:
    """A line list (device tensors are kept alive by this object)."""

    def __init__(self, kind: int, m: int, keep=(), **fields):
        self.kind, self._m, self._keep, self._f = kind, int(m), tuple(keep), fields

    @staticmethod
    def theta_y(theta: torch.Tensor, y: torch.Tensor) -> "Lines":
        th, yy = _dev_f32(theta, "theta"), _dev_f32(y, "y")
        return Lines(KIND_THETA_Y, th.numel(), (th, yy), theta=th.data_ptr(), y=yy.data_ptr())

    @staticmethod
    def points(src: torch.Tensor, dst: torch.Tensor) -> "Lines":
        s, d = _dev_f32(src, "src"), _dev_f32(dst, "dst")
        return Lines(KIND_POINTS, s.numel() // 2, (s, d), src=s.data_ptr(), dst=d.data_ptr())

    @staticmethod
    def parallel(view: torch.Tensor, n_det: int, det0: float, ddet: float) -> "Lines":
        v = _dev_f32(view, "view")
        return Lines(KIND_PARALLEL, v.numel() * int(n_det), (v,), view=v.data_ptr(), n_view=v.numel(),
                     n_det=int(n_det), det0=float(det0), ddet=float(ddet))

    @staticmethod
    def fan(view: torch.Tensor, dso: float, dod: float, n_det: int, det0: float, ddet: float) -> "Lines":
        v = _dev_f32(view, "view")
        return Lines(KIND_FAN, v.numel() * int(n_det), (v,), view=v.data_ptr(), n_view=v.numel(),
                     n_det=int(n_det), det0=float(det0), ddet=float(ddet), dso=float(dso), dod=float(dod))

    @property
    def m(self) -> int:
        return self._m

    def c(self) -> SpLines:
        s = SpLines()
        s.kind = self.kind
        s.m = self._m if self.kind in (KIND_THETA_Y, KIND_POINTS) else 0
        for k, v in self._f.items():
            setattr(s, k, v)
        return s


def spline_project_fwd(grid: Grid, coef: torch.Tensor, lines: Lines, sino: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    c = _dev_f32(coef, "coef")
    if c.numel() != grid.nx * grid.ny:
        raise ValueError("coef must hold ny*nx values")
    if sino is None:
        sino = torch.empty(lines.m, dtype=torch.float32, device=c.device)
    out = _dev_f32(sino, "sino")
    if out.numel() != lines.m or not sino.is_contiguous():
        raise ValueError("sino must be a contiguous tensor of m values")
    g, L = grid.c(), lines.c()
    _check(load().spline_project_fwd(ctypes.byref(g), c.data_ptr(), ctypes.byref(L), out.data_ptr(),
                                     _stream(stream)))
    return sino


def spline_project_adj(grid: Grid, sino: torch.Tensor, lines: Lines, coef_out: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    p = _dev_f32(sino, "sino")
    if p.numel() != lines.m:
        raise ValueError("sino must hold m values")
    if coef_out is None:
        coef_out = torch.empty(grid.ny, grid.nx, dtype=torch.float32, device=p.device)
    out = _dev_f32(coef_out, "coef_out")
    if out.numel() != grid.nx * grid.ny or not coef_out.is_contiguous():
        raise ValueError("coef_out must be a contiguous tensor of ny*nx values")
    g, L = grid.c(), lines.c()
    _check(load().spline_project_adj(ctypes.byref(g), p.data_ptr(), ctypes.byref(L), out.data_ptr(),
                                     _stream(stream)))
    return coef_out


def spline_lines_expand(lines: Lines, device=None, stream=None):
    dev = device or torch.device("cuda")
    th = torch.empty(lines.m, dtype=torch.float32, device=dev)
    yy = torch.empty(lines.m, dtype=torch.float32, device=dev)
    L = lines.c()
    _check(load().spline_lines_expand(ctypes.byref(L), th.data_ptr(), yy.data_ptr(), _stream(stream)))
    return th, yy


def spline_footprint_eval(degree: int, theta: torch.Tensor, yt: torch.Tensor, stream=None,
                          basis: int = BASIS_BSPLINE) -> torch.Tensor:
    th, y = _dev_f32(theta, "theta"), _dev_f32(yt, "yt")
    out = torch.empty_like(th)
    g = SpGrid(1, 1, int(degree), int(basis), 1.0, 0.0, 0.0)
    _check(load().spline_footprint_eval(ctypes.byref(g), th.numel(), th.data_ptr(), y.data_ptr(),
                                        out.data_ptr(), _stream(stream)))
    return out


def spline_visited(grid: Grid, lines: Lines, with_nodes: bool = False, stream=None):
    dev = torch.device("cuda")
    counts = torch.zeros(lines.m, dtype=torch.int32, device=dev)
    g, L = grid.c(), lines.c()
    lib = load()
    _check(lib.spline_visited(ctypes.byref(g), ctypes.byref(L), counts.data_ptr(), None, None,
                              _stream(stream)))
    if not with_nodes:
        return counts
    offs = torch.zeros(lines.m, dtype=torch.int64, device=dev)
    if lines.m > 1:
        offs[1:] = torch.cumsum(counts.to(torch.int64), 0)[:-1]
    total = int(counts.to(torch.int64).sum().item())
    nodes = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    _check(lib.spline_visited(ctypes.byref(g), ctypes.byref(L), counts.data_ptr(), offs.data_ptr(),
                              nodes.data_ptr(), _stream(stream)))
    return counts, offs, nodes[:total]


def sp_release_workspace():
    _check(load().sp_release_workspace())


def sp_version() -> int:
    return int(load().sp_version())


def fp32_peak(packed: bool = False, stream=None) -> tuple[float, float]:
    """Measured FP32 throughput of the current device (sp_fp32_peak): scalar
    or packed (fma.rn.f32x2) FMA chains.  Returns (TFLOP/s, ms per launch)."""
    t, ms = ctypes.c_double(0.0), ctypes.c_float(0.0)
    _check(load().sp_fp32_peak(1 if packed else 0, ctypes.byref(t), ctypes.byref(ms), _stream(stream)))
    return float(t.value), float(ms.value)


class Plan:
    """spline_plan_* wrapper: line records and footprint tables kept on the
    device for repeated projections with one (grid, lines) pair."""

    def __init__(self, grid: Grid, lines: Lines, prepare: bool = True, stream=None, records: bool = False):
        self.grid, self.lines = grid, lines
        self._g, self._L = grid.c(), lines.c()
        h = ctypes.c_void_p()
        _check(load().spline_plan_create(ctypes.byref(self._g), ctypes.byref(self._L), ctypes.byref(h)))
        self._h = h
        if records:
            _check(load().spline_plan_set_records(self._h, 1))
        if prepare:
            self.prepare(stream)

    @property
    def m(self) -> int:
        return self.lines.m

    def prepare(self, stream=None):
        _check(load().spline_plan_prepare(self._h, _stream(stream)))

    def fwd(self, coef: torch.Tensor, sino: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        c = _dev_f32(coef, "coef")
        if c.numel() != self.grid.nx * self.grid.ny:
            raise ValueError("coef must hold ny*nx values")
        if sino is None:
            sino = torch.empty(self.m, dtype=torch.float32, device=c.device)
        if sino.numel() != self.m or not sino.is_contiguous() or sino.dtype != torch.float32:
            raise ValueError("sino must be a contiguous float32 tensor of m values")
        _check(load().spline_plan_fwd(self._h, c.data_ptr(), sino.data_ptr(), _stream(stream)))
        return sino

    def adj(self, sino: torch.Tensor, coef_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        p = _dev_f32(sino, "sino")
        if p.numel() != self.m:
            raise ValueError("sino must hold m values")
        if coef_out is None:
            coef_out = torch.empty(self.grid.ny, self.grid.nx, dtype=torch.float32, device=p.device)
        if coef_out.numel() != self.grid.nx * self.grid.ny or not coef_out.is_contiguous():
            raise ValueError("coef_out must be a contiguous tensor of ny*nx values")
        _check(load().spline_plan_adj(self._h, p.data_ptr(), coef_out.data_ptr(), _stream(stream)))
        return coef_out

    def cgls(self, b: torch.Tensor, iters: int, x0: torch.Tensor | None = None,
             history: bool = True, stream=None):
        """Least squares min ||A x - b|| by CGLS (spline_plan_cgls).

        Returns (x, gamma) with x the last iterate [ny][nx] and gamma the FP64
        history ||A^T (b - A x_k)||^2, k = 0..iters (None if history is False).
        x0 (default zeros) is not modified."""
        bb = _dev_f32(b, "b")
        if bb.numel() != self.m:
            raise ValueError("b must hold m values")
        if x0 is None:
            x = torch.zeros(self.grid.ny, self.grid.nx, dtype=torch.float32, device=bb.device)
        else:
            x = _dev_f32(x0, "x0").clone().reshape(self.grid.ny, self.grid.nx)
        gam = torch.empty(iters + 1, dtype=torch.float64, device=bb.device) if history else None
        _check(load().spline_plan_cgls(self._h, bb.data_ptr(), x.data_ptr(), int(iters),
                                       gam.data_ptr() if history else None, _stream(stream)))
        return x, gam

    def set_paths(self, fwd: int, adj: int):
        """Kernel family per direction: 0 automatic, 1 strip, 2 general; the
        adjoint also 3, the pixel-driven gather."""
        _check(load().spline_plan_set_paths(self._h, int(fwd), int(adj)))

    def autotune(self, coef: torch.Tensor, sino: torch.Tensor, stream=None):
        """Time the kernel families on this data and keep the fastest per
        direction.  Returns (fwd_path, adj_path, [ms fwd strip, fwd general,
        adj strip, adj general, adj gather])."""
        c, p = _dev_f32(coef, "coef"), _dev_f32(sino, "sino")
        f, a = ctypes.c_int32(0), ctypes.c_int32(0)
        ms = (ctypes.c_float * 5)()
        _check(load().spline_plan_autotune(self._h, c.data_ptr(), p.data_ptr(), _stream(stream),
                                           ctypes.byref(f), ctypes.byref(a), ms))
        return f.value, a.value, list(ms)

    def set_records(self, keep: bool = True, stream=None):
        """Keep row records (written by prepare, read by every projection) or
        free them; prepares the plan again when they are kept."""
        _check(load().spline_plan_set_records(self._h, 1 if keep else 0))
        if keep:
            self.prepare(stream)

    def record_bytes(self) -> int:
        """Device bytes of the row records the plan keeps (0: none)."""
        return int(load().spline_plan_record_bytes(self._h))

    def slow_rows(self) -> int:
        """Rows read from global memory because they fell outside the staged window."""
        v = ctypes.c_int64(0)
        _check(load().spline_plan_stats(self._h, ctypes.byref(v)))
        return int(v.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().spline_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """spline_batch_* wrapper: independent instances projected together (one
    CUDA graph per set of data pointers)."""

    def __init__(self, grids, lines, prepare: bool = True, stream=None):
        if len(grids) != len(lines) or not grids:
            raise ValueError("need as many grids as line lists (>= 1)")
        self.grids, self.lines = list(grids), list(lines)
        self._g = (SpGrid * len(grids))(*[g.c() for g in grids])
        self._L = (SpLines * len(lines))(*[L.c() for L in lines])
        h = ctypes.c_void_p()
        _check(load().spline_batch_create(len(grids), self._g, self._L, ctypes.byref(h)))
        self._h = h
        if prepare:
            self.prepare(stream)

    def __len__(self):
        return len(self.grids)

    def prepare(self, stream=None):
        _check(load().spline_batch_prepare(self._h, _stream(stream)))

    @staticmethod
    def _ptrs(ts):
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def fwd(self, coefs, sinos=None, stream=None):
        cs = [_dev_f32(c, "coef") for c in coefs]
        if sinos is None:
            sinos = [torch.empty(L.m, dtype=torch.float32, device=c.device) for L, c in zip(self.lines, cs)]
        self._keep = (cs, sinos)
        _check(load().spline_batch_fwd(self._h, self._ptrs(cs), self._ptrs(sinos), _stream(stream)))
        return sinos

    def adj(self, sinos, coefs_out=None, stream=None):
        ps = [_dev_f32(p, "sino") for p in sinos]
        if coefs_out is None:
            coefs_out = [torch.empty(g.ny, g.nx, dtype=torch.float32, device=p.device) for g, p in zip(self.grids, ps)]
        self._keep = (ps, coefs_out)
        _check(load().spline_batch_adj(self._h, self._ptrs(ps), self._ptrs(coefs_out), _stream(stream)))
        return coefs_out

    def autotune(self, coefs, sinos, stream=None):
        cs = [_dev_f32(c, "coef") for c in coefs]
        ps = [_dev_f32(p, "sino") for p in sinos]
        paths = (ctypes.c_int32 * (2 * len(self)))()
        _check(load().spline_batch_autotune(self._h, self._ptrs(cs), self._ptrs(ps), _stream(stream), paths))
        return [(paths[2 * i], paths[2 * i + 1]) for i in range(len(self))]

    def queued(self, adjoint: bool = False) -> int:
        """Instances that the last recorded forward (or adjoint) graph runs
        through the persistent work-queue kernel."""
        return int(load().spline_batch_queued(self._h, 1 if adjoint else 0))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().spline_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
