"""The pixel-driven gather adjoint (adjoint path 3) against the FP64 oracle
and against the strip scatter: same pairs, same footprint values, summed in
another order, so within FP32 rounding of both."""
import math

import numpy as np
import pytest

import oracle
import workloads
from _geom import device_lines, oracle_lines, rel_l2

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = 1e-5


def _rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / max(float(b.norm()), 1e-300))


CASES = [   # (workload cropped to n x n, degree)
    ("fan512_cubic", 96, 3),
    ("fan512_cubic", 80, 1),
    ("parallel256_cubic", 128, 3),
    ("parallel256_cubic", 72, 2),
]


@pytest.mark.parametrize("base,n,degree", CASES)
def test_gather_adjoint_matches_oracle_and_scatter(base, n, degree):
    W = workloads.crop_workload(workloads.workload(base), n, degree=degree, seed=31)
    grid = sp.Grid(W.n, W.n, W.degree, W.h)
    lines = device_lines(W.geometry, DEV)
    plan = sp.Plan(grid, lines, prepare=True)
    p = torch.randn(lines.m, device=DEV, generator=torch.Generator(DEV).manual_seed(7))
    p[::5] = 0.0
    scatter = plan.adj(p).clone()
    plan.set_paths(0, 3)
    gather = plan.adj(p)
    torch.cuda.synchronize()
    # the strip scatter rounds each contribution to its chunk's fixed-point
    # unit (<= 7e-7 h max|p|); with signed data the node sums cancel, so the
    # two agree to a few 1e-6 here, each within the oracle bar below
    assert _rel(gather, scatter) < 1e-5
    th, yy = oracle_lines(W.geometry)
    ref = oracle.adjoint(oracle.Grid(W.n, W.n, W.degree, W.h), p.cpu().numpy().astype(np.float64), th, yy)
    assert rel_l2(gather.cpu().numpy(), ref) < TOL
    plan.close()


def test_gather_on_an_offset_rectangular_grid():
    # nx != ny, spacing 0.8, centre off the origin: nodes whose support the
    # fan's edge lines only graze, and a tile that hangs over the grid
    nx, ny, h, cx, cy = 77, 90, 0.8, 3.5, -2.25
    view = torch.linspace(0, 2 * math.pi, 121, device=DEV)[:-1].contiguous()
    lines = sp.Lines.fan(view, 160.0, 80.0, 150, -74.5, 0.9)
    grid = sp.Grid(nx, ny, 3, h, cx, cy)
    plan = sp.Plan(grid, lines, prepare=True)
    p = torch.rand(lines.m, device=DEV, generator=torch.Generator(DEV).manual_seed(9))
    plan.set_paths(0, 3)
    got = plan.adj(p).cpu().numpy()
    th, yy = oracle.lines_fan(view.cpu().numpy().astype(np.float64), 160.0, 80.0, 150, -74.5, 0.9)
    ref = oracle.adjoint(oracle.Grid(nx, ny, 3, h, cx, cy), p.cpu().numpy().astype(np.float64), th, yy)
    assert rel_l2(got, ref) < TOL
    plan.close()


def test_gather_path_falls_back_where_it_does_not_apply():
    # degree 0 and the box-spline keep the automatic adjoint under path 3
    W = workloads.crop_workload(workloads.workload("fan512_cubic"), 48, degree=0, seed=3)
    lines = device_lines(W.geometry, DEV)
    for grid in (sp.Grid(W.n, W.n, 0, W.h), sp.Grid(W.n, W.n, 1, W.h, basis=sp.BASIS_BOX3)):
        plan = sp.Plan(grid, lines, prepare=True)
        p = torch.rand(lines.m, device=DEV, generator=torch.Generator(DEV).manual_seed(4))
        a = plan.adj(p).clone()
        plan.set_paths(0, 3)
        b = plan.adj(p)
        torch.cuda.synchronize()
        assert _rel(b, a) < 1e-6
        plan.close()


def test_autotune_times_the_gather():
    W = workloads.crop_workload(workloads.workload("parallel256_cubic"), 64, seed=5)
    grid = sp.Grid(W.n, W.n, W.degree, W.h)
    lines = device_lines(W.geometry, DEV)
    plan = sp.Plan(grid, lines, prepare=True)
    coef = torch.from_numpy(W.coef).to(DEV)
    sino = plan.fwd(coef)
    f, a, ms = plan.autotune(coef, sino)
    assert len(ms) == 5 and ms[4] > 0.0
    assert a in (1, 2, 3)
    back = plan.adj(sino)
    th, yy = oracle_lines(W.geometry)
    ref = oracle.adjoint(oracle.Grid(W.n, W.n, W.degree, W.h), sino.cpu().numpy().astype(np.float64), th, yy)
    assert rel_l2(back.cpu().numpy(), ref) < TOL
    plan.close()
