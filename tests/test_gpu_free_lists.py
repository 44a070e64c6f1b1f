"""Free line lists (THETA_Y, POINTS) on the strip kernels.

Prepare sorts the lines by major axis, direction and offset so that 32
consecutive lines of the order are nearly parallel neighbours; the strip
kernels then take their chunks through that order.  Checked against the FP64
oracle, against the warp-per-line kernels on the same lines, and on the cases
that stress the order: dense random chords (no row may fall outside the
staged windows), a structured scan handed over as a shuffled list, duplicate
lines, lines that miss the grid, ragged chunk counts, lines along the axes,
degree 0, row records and the batch's queue kernel.  Forward outputs are
pre-filled with NaN so that a line the order skipped shows up."""
import math

import numpy as np
import pytest

import oracle
import workloads
from _geom import rel_l2

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = 1e-5


def _phantom(n, seed):
    return np.ascontiguousarray(workloads.ellipse_phantom(n, 8, seed, radius=0.35 * n, axes=(2.0, 0.3 * n)))


def _points(src, dst):
    return sp.Lines.points(torch.from_numpy(np.ascontiguousarray(src)).to(DEV),
                           torch.from_numpy(np.ascontiguousarray(dst)).to(DEV))


def _fwd(plan, coef, m):
    out = torch.full((m,), float("nan"), device=DEV)
    return plan.fwd(coef, out)


def _check_against_oracle_and_general(grid, og, lines, th, yy, coef_np, seed, tol=TOL):
    coef = torch.from_numpy(coef_np).to(DEV)
    plan = sp.Plan(grid, lines, prepare=True)
    sino = _fwd(plan, coef, lines.m)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(sino).all()), "a line of the order was not projected"
    ref = oracle.forward(og, coef_np.astype(np.float64), th, yy)
    assert rel_l2(sino.cpu().numpy(), ref) < tol
    p = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, lines.m).astype(np.float32)).to(DEV)
    back = plan.adj(p).clone()
    ref_b = oracle.adjoint(og, p.cpu().numpy().astype(np.float64), th, yy)
    assert rel_l2(back.cpu().numpy(), ref_b) < tol
    # the warp-per-line kernels on the same lines
    plan.set_paths(2, 2)
    s2 = plan.fwd(coef)
    b2 = plan.adj(p)
    torch.cuda.synchronize()
    assert float((sino - s2).norm() / s2.norm()) < 2e-6
    assert float((back - b2).norm() / b2.norm()) < 1e-5
    plan.close()
    return sino, back


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_random_chords_on_strip_kernels(degree):
    n = 72
    grid = sp.Grid(n, n, degree, 1.0)
    og = oracle.Grid(n, n, degree, 1.0)
    src, dst = workloads.random_lines_circle(20000, 0.75 * n, 40 + degree)
    lines = _points(src, dst)
    th, yy = oracle.lines_points(src.astype(np.float64), dst.astype(np.float64))
    _check_against_oracle_and_general(grid, og, lines, th, yy, _phantom(n, 3 + degree), degree)
    # dense random chords sort into chunks whose windows hold every run
    plan = sp.Plan(grid, lines, prepare=True)
    plan.fwd(torch.from_numpy(_phantom(n, 3)).to(DEV))
    plan.adj(torch.ones(lines.m, device=DEV))
    assert plan.slow_rows() == 0
    plan.close()


def test_theta_y_on_rectangular_offset_grid():
    # random (theta, y) over a non-square grid with its centre off the origin
    # and spacing 0.8: both major axes, lines that miss the grid
    nx, ny, h, cx, cy = 61, 44, 0.8, 2.5, -1.75
    rng = np.random.default_rng(12)
    m = 9001
    th = rng.uniform(0.0, 2.0 * math.pi, m).astype(np.float32)
    yy = rng.uniform(-40.0, 40.0, m).astype(np.float32)
    lines = sp.Lines.theta_y(torch.from_numpy(th).to(DEV), torch.from_numpy(yy).to(DEV))
    for degree in (1, 3):
        grid = sp.Grid(nx, ny, degree, h, cx, cy)
        og = oracle.Grid(nx, ny, degree, h, cx, cy)
        coef = np.ascontiguousarray(workloads.ellipse_phantom(max(nx, ny), 8, 9, radius=20.0, axes=(2.0, 14.0))[:ny, :nx])
        _check_against_oracle_and_general(grid, og, lines, th.astype(np.float64), yy.astype(np.float64), coef, 5)


def test_shuffled_fan_scan_as_point_pairs():
    # a fan scan handed over as a shuffled list of (source, detector bin)
    # point pairs: the sort has to rebuild the view structure
    n = 64
    views = np.linspace(0, 2 * math.pi, 90, endpoint=False)
    dso, dod, n_det, ddet = 120.0, 60.0, 96, 1.0
    det0 = -0.5 * (n_det - 1) * ddet
    b = np.repeat(views, n_det)
    j = np.tile(np.arange(n_det), views.size)
    srcs = np.stack([dso * np.cos(b), dso * np.sin(b)], 1)
    t = det0 + j * ddet
    dsts = np.stack([-dod * np.cos(b) - t * np.sin(b), -dod * np.sin(b) + t * np.cos(b)], 1)
    perm = np.random.default_rng(3).permutation(b.size)
    src, dst = srcs[perm].astype(np.float32), dsts[perm].astype(np.float32)
    grid, og = sp.Grid(n, n, 3, 1.0), oracle.Grid(n, n, 3, 1.0)
    lines = _points(src, dst)
    th, yy = oracle.lines_points(src.astype(np.float64), dst.astype(np.float64))
    _check_against_oracle_and_general(grid, og, lines, th, yy, _phantom(n, 8), 6)
    plan = sp.Plan(grid, lines, prepare=True)
    plan.fwd(torch.from_numpy(_phantom(n, 8)).to(DEV))
    assert plan.slow_rows() == 0
    plan.close()


@pytest.mark.parametrize("m", [1, 31, 33, 65])
def test_ragged_and_tiny_lists(m):
    n = 40
    src, dst = workloads.random_lines_circle(m, 0.75 * n, 100 + m)
    grid, og = sp.Grid(n, n, 2, 1.0), oracle.Grid(n, n, 2, 1.0)
    lines = _points(src, dst)
    th, yy = oracle.lines_points(src.astype(np.float64), dst.astype(np.float64))
    _check_against_oracle_and_general(grid, og, lines, th, yy, _phantom(n, 2), 7)


def test_duplicates_misses_and_axis_lines():
    # 300 copies of one chord, lines far outside the grid, lines exactly along
    # both axes through nodes and between them, and random chords
    n = 48
    rng = np.random.default_rng(21)
    th = [np.full(300, 0.61), np.array([0.2, 1.3, 2.9]), np.zeros(40), np.full(40, math.pi / 2),
          np.full(20, math.pi), rng.uniform(0, 2 * math.pi, 500)]
    yy = [np.full(300, 3.3), np.array([80.0, -75.0, 200.0]), np.arange(40) - 20.0,
          np.arange(40) * 0.5 - 10.0, np.arange(20) - 9.5, rng.uniform(-30, 30, 500)]
    th = np.concatenate(th).astype(np.float32)
    yy = np.concatenate(yy).astype(np.float32)
    perm = rng.permutation(th.size)
    th, yy = th[perm], yy[perm]
    lines = sp.Lines.theta_y(torch.from_numpy(th).to(DEV), torch.from_numpy(yy).to(DEV))
    for degree in (1, 3):
        grid, og = sp.Grid(n, n, degree, 1.0), oracle.Grid(n, n, degree, 1.0)
        sino, _ = _check_against_oracle_and_general(grid, og, lines, th.astype(np.float64),
                                                    yy.astype(np.float64), _phantom(n, 4), 8)
        s = sino.cpu().numpy()
        dup = s[np.nonzero(perm < 300)[0]]
        assert np.all(dup == dup[0])          # copies of one line: the same sum, bit for bit
        miss = s[np.nonzero((perm >= 300) & (perm < 303))[0]]
        assert np.all(miss == 0.0)


def test_degree0_free_list_on_strip_kernels():
    # degree 0 stays on the warp-per-line kernels unless asked; asked, the
    # strip kernels take the sorted list too (axis-aligned lines included)
    n = 40
    rng = np.random.default_rng(5)
    th = np.concatenate([rng.uniform(0, math.pi, 3000), np.zeros(30), np.full(30, math.pi / 2)]).astype(np.float32)
    yy = np.concatenate([rng.uniform(-28, 28, 3000), np.arange(30) - 14.5, np.arange(30) - 15.0]).astype(np.float32)
    lines = sp.Lines.theta_y(torch.from_numpy(th).to(DEV), torch.from_numpy(yy).to(DEV))
    grid, og = sp.Grid(n, n, 0, 1.0), oracle.Grid(n, n, 0, 1.0)
    coef_np = _phantom(n, 6)
    coef = torch.from_numpy(coef_np).to(DEV)
    plan = sp.Plan(grid, lines, prepare=True)
    plan.set_paths(1, 1)
    sino = _fwd(plan, coef, lines.m)
    p = torch.from_numpy(rng.uniform(-1, 1, lines.m).astype(np.float32)).to(DEV)
    back = plan.adj(p)
    thd, yyd = th.astype(np.float64), yy.astype(np.float64)
    assert rel_l2(sino.cpu().numpy(), oracle.forward(og, coef_np.astype(np.float64), thd, yyd)) < TOL
    assert rel_l2(back.cpu().numpy(), oracle.adjoint(og, p.cpu().numpy().astype(np.float64), thd, yyd)) < TOL
    plan.close()


def test_free_list_records_and_one_shot():
    # the one-shot entry points sort the same way (deterministic order): the
    # plan's forward, with or without kept records, equals them bit for bit
    n = 64
    src, dst = workloads.random_lines_circle(12000, 0.75 * n, 9)
    grid = sp.Grid(n, n, 3, 1.0)
    lines = _points(src, dst)
    coef = torch.from_numpy(_phantom(n, 1)).to(DEV)
    one = sp.spline_project_fwd(grid, coef, lines)
    plan = sp.Plan(grid, lines, prepare=True)
    a = plan.fwd(coef).clone()
    plan_r = sp.Plan(grid, lines, prepare=True, records=True)
    assert plan_r.record_bytes() > 0
    b = plan_r.fwd(coef).clone()
    p = torch.randn(lines.m, device=DEV, generator=torch.Generator(DEV).manual_seed(2))
    back_one = sp.spline_project_adj(grid, p, lines)
    back_r = plan_r.adj(p)
    torch.cuda.synchronize()
    assert torch.equal(one, a) and torch.equal(one, b)
    assert float((back_r - back_one).norm() / back_one.norm()) < 1e-6
    plan.close()
    plan_r.close()


def test_batch_queues_free_lists():
    n = 48
    grids, lines, coefs = [], [], []
    for k, deg in enumerate((3, 1, 2)):
        src, dst = workloads.random_lines_circle(3000 + 1000 * k, 0.75 * n, 60 + k)
        grids.append(sp.Grid(n, n, deg, 1.0))
        lines.append(_points(src, dst))
        coefs.append(torch.from_numpy(_phantom(n, 10 + k)).to(DEV))
    batch = sp.Batch(grids, lines)
    plans = [sp.Plan(g, L) for g, L in zip(grids, lines)]
    sinos = batch.fwd(coefs)
    backs = batch.adj(sinos)
    assert batch.queued(False) == 3 and batch.queued(True) == 3
    for s, bk, p, c in zip(sinos, backs, plans, coefs):
        assert torch.equal(s, p.fwd(c))
        ref = p.adj(s)
        assert float((bk - ref).norm() / ref.norm()) < 1e-6
    batch.close()
    for p in plans:
        p.close()
