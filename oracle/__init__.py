"""FP64 CPU oracle of the spline x-ray projector.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or calls it, and
this package never imports the product package.

The arithmetic lives in ``spline_oracle.c`` (plain C, double precision, built
with gcc by :func:`build`); this module only marshals numpy arrays through
ctypes.  What each function computes, with the passage of the paper it
follows:

* :func:`bspline`      centred B-spline beta^n, truncated-power definition
                       (Sec. III.C, beta^n of [unser1993b]).
* :func:`footprint`    phi_theta(y): Prop. 1 / eq. xsa, the convolution of the
                       two rescaled B-splines, integrated exactly piece by piece
                       with Gauss-Legendre; a Dirac replaces a zero scale.
* :func:`box3`, :func:`footprint_box`
                       the 3-direction box-spline of Sec. III.D from its
                       definition (density of a sum of three uniform
                       segments) and its exact line integral (piecewise
                       linear along the line, trapezoid rule per piece).
* :func:`lines_parallel`, :func:`lines_fan`, :func:`lines_points`
                       geometry -> (theta, y) with theta^perp = (sin, -cos)
                       (eq. rayparam).
* :func:`forward`      p_m = h sum_k c_k phi_{theta_m}((y_m - <x_k, theta^perp>)/h)
                       (eq. xrtbasis, discretised operator of Sec. IV.A).
* :func:`adjoint`, :func:`adjoint_pixels`
                       c'_k = h sum_m p_m phi_{theta_m}(...) (the transpose,
                       Sec. II.B "exactly matched").
* :func:`visited`      the nonzero pairs {(m, k): |y~| < w}.
* :func:`alg2_line`    Algorithm 2 with K neighbours (Lemma 1), cross-check only.
* :func:`siddon_line`  classical Siddon intersection lengths (degree 0).

Pins (tests/test_oracle_*.py) tie each function to values fixed by the paper or
by mathematics outside this code: B-spline values, the theta = 0 profile, the
printed n = 1 footprint, brute-force quadrature along the line with an
independent B-spline, Siddon at degree 0, mass conservation, symmetry and the
adjoint identity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "spline_oracle.c"
_OUT_DIR = _HERE / "_build"
_LIB_PATH = _OUT_DIR / "liboracle.so"
_lib = None


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("basis", ctypes.c_int32),
                ("h", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


def build(force: bool = False) -> Path:
    """Compile spline_oracle.c with gcc (OpenMP if available) into oracle/_build."""
    _OUT_DIR.mkdir(exist_ok=True)
    if _LIB_PATH.exists() and not force and _LIB_PATH.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB_PATH
    tmp = _OUT_DIR / f"liboracle.{os.getpid()}.so"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", str(_SRC), "-o", str(tmp), "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(str(_LIB_PATH))
    d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
    P = ctypes.c_void_p
    lib.orc_bspline.restype = d
    lib.orc_bspline.argtypes = [ctypes.c_int, d]
    lib.orc_footprint.restype = d
    lib.orc_footprint.argtypes = [ctypes.c_int, d, d, d]
    lib.orc_support_halfwidth.restype = d
    lib.orc_support_halfwidth.argtypes = [ctypes.c_int, d, d]
    lib.orc_box3.restype = d
    lib.orc_box3.argtypes = [d, d]
    lib.orc_footprint_box.restype = d
    lib.orc_footprint_box.argtypes = [d, d, d]
    lib.orc_support_halfwidth_box.restype = d
    lib.orc_support_halfwidth_box.argtypes = [d, d]
    lib.orc_lines_parallel.argtypes = [i32, P, i32, d, d, P, P]
    lib.orc_lines_fan.argtypes = [i32, P, d, d, i32, d, d, P, P]
    lib.orc_lines_points.argtypes = [i64, P, P, P, P]
    lib.orc_forward.argtypes = [ctypes.POINTER(_Grid), P, i64, P, P, P, i32, i32]
    lib.orc_adjoint.argtypes = [ctypes.POINTER(_Grid), P, i64, P, P, P, i32]
    lib.orc_adjoint_pixels.argtypes = [ctypes.POINTER(_Grid), P, i64, P, P, i64, P, P, i32]
    lib.orc_visited.argtypes = [ctypes.POINTER(_Grid), i64, P, P, i32, P, P, P, P]
    lib.orc_alg2_line.restype = i64
    lib.orc_alg2_line.argtypes = [ctypes.POINTER(_Grid), P, d, d, i32, P, P, P]
    lib.orc_siddon_line.restype = d
    lib.orc_siddon_line.argtypes = [ctypes.POINTER(_Grid), P, d, d]
    lib.orc_max_threads.restype = i32
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _grid(nx, ny, degree, h=1.0, cx=0.0, cy=0.0, basis=0) -> _Grid:
    return _Grid(int(nx), int(ny), int(degree), int(basis), float(h), float(cx), float(cy))


class Grid:
    """Coefficient grid: nx x ny nodes, spacing h, centred at (cx, cy).

    Node (i, j) sits at (cx + (i - (nx-1)/2) h, cy + (j - (ny-1)/2) h);
    coefficient arrays are [ny][nx] (row j, column i fastest).  basis 0 is the
    tensor-product B-spline of the given degree, basis 1 the 3-direction
    box-spline (degree ignored)."""

    def __init__(self, nx, ny, degree, h=1.0, cx=0.0, cy=0.0, basis=0):
        self.nx, self.ny, self.degree = int(nx), int(ny), int(degree)
        self.h, self.cx, self.cy = float(h), float(cx), float(cy)
        self.basis = int(basis)

    def _c(self) -> _Grid:
        return _grid(self.nx, self.ny, self.degree, self.h, self.cx, self.cy, self.basis)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def bspline(n: int, x: float) -> float:
    return float(_load().orc_bspline(int(n), float(x)))


def footprint(n: int, theta: float, yt: float) -> float:
    """phi_theta(yt) on the unit grid (cos/sin taken in double from theta)."""
    return float(_load().orc_footprint(int(n), float(np.cos(theta)), float(np.sin(theta)), float(yt)))


def footprint_cs(n: int, ct: float, st: float, yt: float) -> float:
    return float(_load().orc_footprint(int(n), float(ct), float(st), float(yt)))


def box3(x1: float, x2: float) -> float:
    """3-direction box-spline (directions e1, e2, e1 + e2; Sec. III.D) at (x1, x2)."""
    return float(_load().orc_box3(float(x1), float(x2)))


def footprint_box(theta: float, yt: float) -> float:
    """x-ray transform of the box-spline along theta at offset yt."""
    return float(_load().orc_footprint_box(float(np.cos(theta)), float(np.sin(theta)), float(yt)))


def footprint_box_cs(ct: float, st: float, yt: float) -> float:
    return float(_load().orc_footprint_box(float(ct), float(st), float(yt)))


def support_halfwidth_box(theta: float) -> float:
    return float(_load().orc_support_halfwidth_box(float(np.cos(theta)), float(np.sin(theta))))


def support_halfwidth(n: int, theta: float) -> float:
    return float(_load().orc_support_halfwidth(int(n), float(np.cos(theta)), float(np.sin(theta))))


def lines_parallel(angles, n_det: int, det0: float, ddet: float):
    ang = _f64(angles)
    m = ang.size * int(n_det)
    th, y = np.empty(m), np.empty(m)
    _load().orc_lines_parallel(ang.size, _ptr(ang), int(n_det), float(det0), float(ddet), _ptr(th), _ptr(y))
    return th, y


def lines_fan(beta, dso: float, dod: float, n_det: int, det0: float, ddet: float):
    b = _f64(beta)
    m = b.size * int(n_det)
    th, y = np.empty(m), np.empty(m)
    _load().orc_lines_fan(b.size, _ptr(b), float(dso), float(dod), int(n_det), float(det0), float(ddet),
                          _ptr(th), _ptr(y))
    return th, y


def lines_points(src, dst):
    s, d = _f64(src).reshape(-1, 2), _f64(dst).reshape(-1, 2)
    m = s.shape[0]
    th, y = np.empty(m), np.empty(m)
    _load().orc_lines_points(m, _ptr(s), _ptr(d), _ptr(th), _ptr(y))
    return th, y


def forward(grid: Grid, coef, theta, y, brute: bool = False, threads: int = 0) -> np.ndarray:
    c = _f64(coef).reshape(grid.ny, grid.nx)
    th, yy = _f64(theta).ravel(), _f64(y).ravel()
    out = np.empty(th.size)
    g = grid._c()
    _load().orc_forward(ctypes.byref(g), _ptr(c), th.size, _ptr(th), _ptr(yy), _ptr(out),
                        int(bool(brute)), int(threads))
    return out


def adjoint(grid: Grid, sino, theta, y, threads: int = 0) -> np.ndarray:
    p = _f64(sino).ravel()
    th, yy = _f64(theta).ravel(), _f64(y).ravel()
    out = np.empty(grid.nx * grid.ny)
    g = grid._c()
    _load().orc_adjoint(ctypes.byref(g), _ptr(p), th.size, _ptr(th), _ptr(yy), _ptr(out), int(threads))
    return out.reshape(grid.ny, grid.nx)


def adjoint_pixels(grid: Grid, sino, theta, y, pix, threads: int = 0) -> np.ndarray:
    p = _f64(sino).ravel()
    th, yy = _f64(theta).ravel(), _f64(y).ravel()
    px = np.ascontiguousarray(np.asarray(pix, dtype=np.int64).ravel())
    out = np.empty(px.size)
    g = grid._c()
    _load().orc_adjoint_pixels(ctypes.byref(g), _ptr(p), th.size, _ptr(th), _ptr(yy), px.size, _ptr(px),
                               _ptr(out), int(threads))
    return out


def visited(grid: Grid, theta, y, brute: bool = False, with_index: bool = False):
    """Per-line counts of nonzero pairs; optionally the CSR node lists and
    the smallest distance ||y~| - w| seen over the tested pairs."""
    th, yy = _f64(theta).ravel(), _f64(y).ravel()
    counts = np.zeros(th.size, dtype=np.int64)
    gap = ctypes.c_double(0.0)
    g = grid._c()
    lib = _load()
    lib.orc_visited(ctypes.byref(g), th.size, _ptr(th), _ptr(yy), int(bool(brute)), _ptr(counts),
                    None, None, ctypes.byref(gap))
    if not with_index:
        return counts, gap.value
    offs = np.zeros(th.size + 1, dtype=np.int64)
    np.cumsum(counts, out=offs[1:])
    idx = np.empty(int(offs[-1]), dtype=np.int64)
    lib.orc_visited(ctypes.byref(g), th.size, _ptr(th), _ptr(yy), int(bool(brute)), _ptr(counts),
                    _ptr(offs), _ptr(idx), None)
    return counts, gap.value, offs, idx


def alg2_line(grid: Grid, coef, theta: float, y: float, K: int):
    c = _f64(coef).reshape(grid.ny, grid.nx)
    mark = np.zeros(grid.nx * grid.ny, dtype=np.uint8)
    cand = np.empty(grid.nx * grid.ny, dtype=np.int64)
    val = ctypes.c_double(0.0)
    g = grid._c()
    nc = _load().orc_alg2_line(ctypes.byref(g), _ptr(c), float(theta), float(y), int(K), _ptr(mark),
                               _ptr(cand), ctypes.byref(val))
    return cand[:nc].copy(), val.value


def siddon_line(grid: Grid, coef, theta: float, y: float) -> float:
    c = _f64(coef).reshape(grid.ny, grid.nx)
    g = grid._c()
    return float(_load().orc_siddon_line(ctypes.byref(g), _ptr(c), float(theta), float(y)))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
