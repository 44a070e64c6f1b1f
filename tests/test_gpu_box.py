"""Parity of the CUDA projector with the 3-direction box-spline basis
(Sec. III.D) against the FP64 oracle: its footprint table, forward and
adjoint on every line-list kind (the strip kernels by default, free lists
through their sorted order), the adjoint identity, the
visited set, and the 256 x 256 fan geometry on sampled lines.  Same bar as
the B-spline projector: relative L2 <= 1e-5."""
import math

import numpy as np
import pytest

import oracle
import workloads
from _geom import device_lines, oracle_lines, rel_l2

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda"


def _grid(n, h=1.0, cx=0.0, cy=0.0, ny=None):
    ny = n if ny is None else ny
    return (sp.Grid(n, ny, 1, h, cx, cy, basis=sp.BASIS_BOX3),
            oracle.Grid(n, ny, 1, h, cx, cy, basis=1))


def test_box_footprint_table_matches_oracle():
    rng = np.random.default_rng(901)
    special = [0.0, 1e-7, 1e-6, 1e-4, 1e-2, math.pi / 4, math.pi / 4 + 1e-6, math.pi / 4 - 1e-5,
               math.atan(0.5), math.pi / 2, math.pi / 2 + 1e-6, 3 * math.pi / 4, 3 * math.pi / 4 + 1e-6,
               math.pi - 1e-5, 2.0, -0.3]
    th = np.concatenate([rng.uniform(0, 2 * math.pi, 300), special]).astype(np.float32)
    th = np.repeat(th, 40)
    t64 = th.astype(np.float64)
    w = 0.5 * (np.abs(np.sin(t64)) + np.abs(np.cos(t64)) + np.abs(np.sin(t64) - np.cos(t64)))
    yt = (rng.uniform(-1.1, 1.1, th.size) * w).astype(np.float32)
    got = sp.spline_footprint_eval(1, torch.from_numpy(th).to(DEV), torch.from_numpy(yt).to(DEV),
                                   basis=sp.BASIS_BOX3).cpu().numpy()
    ref = np.array([oracle.footprint_box(float(t), float(y)) for t, y in zip(th, yt)])
    err = np.abs(got.astype(np.float64) - ref)
    assert err.max() < 2e-6, f"max abs error {err.max():.3e} at theta {th[err.argmax()]}"


def _small_geometry(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "parallel":
        return workloads.Geometry("parallel", view_angle=np.sort(rng.uniform(0, math.pi, 37)).astype(np.float32),
                                  n_det=53, det0=-27.3, ddet=1.03)
    if kind == "fan":
        return workloads.Geometry("fan", view_angle=np.linspace(0, 2 * math.pi, 41, endpoint=False).astype(np.float32),
                                  n_det=61, det0=-30.0 * 1.1, ddet=1.1, dso=80.0, dod=40.0)
    src, dst = workloads.random_lines_circle(1500, 0.75 * n, seed)
    return workloads.Geometry("points", src=src, dst=dst)


@pytest.mark.parametrize("kind", ["parallel", "fan", "points"])
def test_box_forward_and_adjoint_small(kind):
    N, NY = 37, 29
    g, og = _grid(N, h=0.9, cx=0.35, cy=-0.2, ny=NY)
    geo = _small_geometry(kind, N, 910)
    coef = np.ascontiguousarray(workloads.ellipse_phantom(N, 8, 41, radius=0.35 * N, axes=(2.0, 0.3 * N))[:NY, :])
    lines = device_lines(geo, DEV)
    th, yy = oracle_lines(geo)
    sino = sp.spline_project_fwd(g, torch.from_numpy(coef).to(DEV), lines).cpu().numpy()
    assert rel_l2(sino, oracle.forward(og, coef, th, yy)) < TOL
    p = np.random.default_rng(9).uniform(-1, 1, th.size).astype(np.float32)
    back = sp.spline_project_adj(g, torch.from_numpy(p).to(DEV), lines).cpu().numpy()
    assert rel_l2(back, oracle.adjoint(og, p, th, yy)) < TOL


def test_box_theta_y_lines_special_angles():
    # axis-aligned and diagonal directions, where one box width vanishes
    N = 24
    g, og = _grid(N)
    base = [0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, math.pi, 1e-6, math.pi / 4 + 1e-6, 0.7]
    th = np.repeat(np.array(base, dtype=np.float32), 31)
    y = np.tile(np.linspace(-15.5, 15.5, 31), len(base)).astype(np.float32)
    coef = workloads.ellipse_phantom(N, 6, 42, radius=8.0, axes=(2.0, 7.0))
    lines = sp.Lines.theta_y(torch.from_numpy(th).to(DEV), torch.from_numpy(y).to(DEV))
    sino = sp.spline_project_fwd(g, torch.from_numpy(coef).to(DEV), lines).cpu().numpy()
    ref = oracle.forward(og, coef, th.astype(np.float64), y.astype(np.float64))
    assert rel_l2(sino, ref) < TOL


def test_box_adjoint_identity_and_visited():
    g, og = _grid(48)
    geo = _small_geometry("fan", 48, 77)
    lines = device_lines(geo, DEV)
    gen = torch.Generator(device=DEV).manual_seed(3)
    x = torch.rand(48, 48, device=DEV, generator=gen) - 0.5
    y = torch.rand(lines.m, device=DEV, generator=gen) - 0.5
    Ax = sp.spline_project_fwd(g, x, lines)
    Aty = sp.spline_project_adj(g, y, lines)
    lhs = float(torch.dot(Ax.double(), y.double()))
    rhs = float(torch.dot(x.double().ravel(), Aty.double().ravel()))
    assert abs(lhs - rhs) <= 1e-6 * float(Ax.double().norm() * y.double().norm())
    # visited set: identical counts where no pair is within 1e-5 of the support edge
    th, yy = oracle_lines(geo)
    counts, gap = oracle.visited(og, th, yy)
    got = sp.spline_visited(g, lines).cpu().numpy()
    if gap > 1e-5:
        assert np.array_equal(got, counts)
    else:
        assert np.abs(got.astype(np.int64) - counts).max() <= 2


def test_box_fan256_sampled():
    wl = workloads.workload("fan256_cubic")
    g, og = _grid(wl.n, wl.h)
    lines = device_lines(wl.geometry, DEV)
    th, yy = oracle_lines(wl.geometry)
    sino = sp.spline_project_fwd(g, torch.from_numpy(wl.coef).to(DEV), lines).cpu().numpy()
    idx = np.random.default_rng(5).choice(th.size, 2000, replace=False)
    ref = oracle.forward(og, wl.coef, th[idx], yy[idx])
    assert rel_l2(sino[idx], ref) < TOL
    plan = sp.Plan(g, lines)
    assert plan.slow_rows() == 0
