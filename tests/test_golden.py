"""Golden fixtures (tests/golden/, written by tests/golden/make_golden.py from
the FP64 oracle alone): the oracle still reproduces them, their theta = 0
rows agree with scipy's B-spline (the Dirac case of Prop. 1), and the CUDA
path matches them (visited pairs exactly, footprint values within 2e-6;
1e-5 at degree 0)."""
import os

import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle
import workloads

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _visited():
    total, per_view = None, {}
    for line in open(os.path.join(GOLD, "visited_parallel64_linear.txt")):
        if line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "total":
            total = int(f[1])
        else:
            per_view[int(f[1])] = int(f[2])
    return total, np.array([per_view[v] for v in range(len(per_view))], dtype=np.int64)


def _footprints():
    rows = []
    for line in open(os.path.join(GOLD, "footprint_values.txt")):
        if line.startswith("#"):
            continue
        n, th, y, v = line.split()
        rows.append((int(n), float(th), float(y), float(v)))
    return rows


def _geometry():
    wl = workloads.workload("parallel64_linear")
    geo = wl.geometry
    th, yy = oracle.lines_parallel(geo.view_angle.astype(np.float64), geo.n_det, geo.det0, geo.ddet)
    return wl, geo, th, yy


def test_golden_visited_counts_from_oracle():
    total, per_view = _visited()
    assert total == 938120 and per_view.sum() == total and per_view.size == 90
    wl, geo, th, yy = _geometry()
    counts, _ = oracle.visited(oracle.Grid(wl.n, wl.n, wl.degree, wl.h), th, yy, brute=False)
    assert np.array_equal(counts.reshape(90, 96).sum(axis=1), per_view)


def test_golden_footprints_from_oracle_and_scipy():
    for n, th, y, v in _footprints():
        assert oracle.footprint(n, th, y) == pytest.approx(v, rel=1e-14, abs=1e-15)
        if th == 0.0 and not (n == 0 and abs(abs(y) - 0.5) < 1e-12):
            knots = np.arange(n + 2, dtype=float) - 0.5 * (n + 1)
            ref = BSpline.basis_element(knots, extrapolate=False)(y)
            ref = 0.0 if np.isnan(ref) else float(ref)
            assert v == pytest.approx(ref, abs=1e-14)


@pytest.mark.gpu
def test_golden_against_cuda_path():
    torch = pytest.importorskip("torch")
    sp = pytest.importorskip("paper_2503_20907_gb300")
    from _geom import device_lines
    total, per_view = _visited()
    wl, geo, th, yy = _geometry()
    g = sp.Grid(wl.n, wl.n, wl.degree, wl.h)
    counts = sp.spline_visited(g, device_lines(geo, "cuda")).cpu().numpy().astype(np.int64)
    assert int(counts.sum()) == total
    assert np.array_equal(counts.reshape(90, 96).sum(axis=1), per_view)
    rows = _footprints()
    for n in range(4):
        sel = [r for r in rows if r[0] == n]
        tt = torch.tensor([r[1] for r in sel], dtype=torch.float32, device="cuda")
        yy_ = torch.tensor([r[2] for r in sel], dtype=torch.float32, device="cuda")
        got = sp.spline_footprint_eval(n, tt, yy_).cpu().numpy().astype(np.float64)
        # the kernel sees theta and y rounded to float32: compare with the
        # oracle at those inputs, and with the stored value where exact
        ref = np.array([oracle.footprint(n, float(np.float32(r[1])), float(np.float32(r[2]))) for r in sel])
        # degree 0: ramps of slope 1/(a b) turn the float32 rounding of a
        # and b into up to ~1e-5 in value (as in the footprint parity test)
        assert np.max(np.abs(got - ref)) < (1e-5 if n == 0 else 2e-6)
        exact = [i for i, r in enumerate(sel) if float(np.float32(r[1])) == r[1] and float(np.float32(r[2])) == r[2]]
        assert np.max(np.abs(got[exact] - np.array([sel[i][3] for i in exact]))) < 2e-6
