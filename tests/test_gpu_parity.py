"""Parity of the CUDA projector (through the C ABI) with the FP64 oracle.

Bar: relative L2 error <= 1e-5 per sinogram / per backprojected image in FP32,
and the identical set of nonzero (line, node) pairs on the 64 x 64 linear
workload.  Inputs are the seeded generators of `workloads`; each side expands
the geometry itself."""
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


def _grid(n, degree, h=1.0, cx=0.0, cy=0.0, ny=None):
    ny = n if ny is None else ny
    return sp.Grid(n, ny, degree, h, cx, cy), oracle.Grid(n, ny, degree, h, cx, cy)


# ------------------------------------------------------------------ footprint
@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_footprint_table_matches_oracle(n):
    rng = np.random.default_rng(300 + n)
    th = np.concatenate([rng.uniform(0, 2 * math.pi, 300),
                         [0.0, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, math.pi / 4, math.pi / 2, 0.3,
                          math.pi / 4 + 1e-6, math.pi - 1e-5, 2.0]]).astype(np.float32)
    th = np.repeat(th, 40)
    w = 0.5 * (n + 1) * (np.abs(np.cos(th.astype(np.float64))) + np.abs(np.sin(th.astype(np.float64))))
    yt = (rng.uniform(-1.1, 1.1, th.size) * w).astype(np.float32)
    got = sp.spline_footprint_eval(n, torch.from_numpy(th).to(DEV), torch.from_numpy(yt).to(DEV)).cpu().numpy()
    ref = np.array([oracle.footprint(n, float(t), float(y)) for t, y in zip(th, yt)])
    err = np.abs(got.astype(np.float64) - ref)
    tol = 2e-6
    if n == 0:
        # Degree 0 has ramps of slope 1/(a b): the float32 rounding of a and b
        # moves them by ~1e-8, i.e. up to ~1e-5 in value once b > 1e-3.
        a = np.maximum(np.abs(np.cos(th.astype(np.float64))), np.abs(np.sin(th.astype(np.float64))))
        b = np.minimum(np.abs(np.cos(th.astype(np.float64))), np.abs(np.sin(th.astype(np.float64))))
        err = err[b > 1e-3]
        tol = 1e-5
    assert err.max() < tol, f"max abs error {err.max():.3e}"


# ------------------------------------------------------------------ small parity
CASES = [
    ("parallel", 0), ("parallel", 1), ("parallel", 2), ("parallel", 3),
    ("fan", 0), ("fan", 1), ("fan", 2), ("fan", 3),
    ("points", 1), ("points", 3),
]


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


@pytest.mark.parametrize("kind,n", CASES)
def test_forward_and_adjoint_small(kind, n):
    N, NY = 37, 29   # several tiles of rows and a ragged, non-square grid
    g, og = _grid(N, n, h=0.9, cx=0.35, cy=-0.2, ny=NY)
    geo = _small_geometry(kind, N, 500 + 7 * n)
    coef = workloads.ellipse_phantom(N, 8, 40 + n, radius=0.35 * N, axes=(2.0, 0.3 * N))[:NY, :]
    coef = np.ascontiguousarray(coef)
    lines = device_lines(geo, DEV)
    th, yy = oracle_lines(geo)
    sino = sp.spline_project_fwd(g, torch.from_numpy(coef).to(DEV), lines).cpu().numpy()
    ref = oracle.forward(og, coef, th, yy)
    assert rel_l2(sino, ref) < TOL
    p = np.random.default_rng(9).uniform(-1, 1, th.size).astype(np.float32)
    back = sp.spline_project_adj(g, torch.from_numpy(p).to(DEV), lines).cpu().numpy()
    ref_b = oracle.adjoint(og, p, th, yy)
    assert rel_l2(back, ref_b) < TOL


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_adjoint_identity_gpu(n):
    g, _ = _grid(48, n)
    geo = _small_geometry("fan", 48, 77)
    lines = device_lines(geo, DEV)
    gen = torch.Generator(device=DEV).manual_seed(n)
    x = torch.rand(48, 48, device=DEV, generator=gen) - 0.5
    y = torch.rand(lines.m, device=DEV, generator=gen) - 0.5
    Ax = sp.spline_project_fwd(g, x, lines)
    Aty = sp.spline_project_adj(g, y, lines)
    lhs = float(torch.dot(Ax.double(), y.double()))
    rhs = float(torch.dot(x.double().ravel(), Aty.double().ravel()))
    assert abs(lhs - rhs) <= 1e-6 * float(Ax.double().norm() * y.double().norm())


# ------------------------------------------------------------------ 64 x 64 linear workload
def test_parallel64_linear_full():
    wl = workloads.workload("parallel64_linear")
    g, og = _grid(wl.n, wl.degree, wl.h)
    lines = device_lines(wl.geometry, DEV)
    th, yy = oracle_lines(wl.geometry)
    sino = sp.spline_project_fwd(g, torch.from_numpy(wl.coef).to(DEV), lines).cpu().numpy()
    ref = oracle.forward(og, wl.coef, th, yy, brute=True)
    assert rel_l2(sino, ref) < TOL
    back = sp.spline_project_adj(g, torch.from_numpy(sino).to(DEV), lines).cpu().numpy()
    assert rel_l2(back, oracle.adjoint(og, sino.astype(np.float64), th, yy)) < TOL


def test_parallel64_linear_visited_set_identical():
    wl = workloads.workload("parallel64_linear")
    g, og = _grid(wl.n, wl.degree, wl.h)
    lines = device_lines(wl.geometry, DEV)
    th, yy = oracle_lines(wl.geometry)
    rc, gap, roffs, ridx = oracle.visited(og, th, yy, brute=True, with_index=True)
    assert gap > 1e-5   # no pair within FP32 reach of the support boundary
    counts, offs, nodes = sp.spline_visited(g, lines, with_nodes=True)
    counts, offs, nodes = counts.cpu().numpy(), offs.cpu().numpy(), nodes.cpu().numpy()
    assert np.array_equal(counts.astype(np.int64), rc)
    for m in range(th.size):
        a = np.sort(nodes[offs[m]:offs[m] + counts[m]].astype(np.int64))
        b = np.sort(ridx[roffs[m]:roffs[m + 1]])
        assert np.array_equal(a, b), m


# ------------------------------------------------------------------ full size, sampled
def test_fan512_cubic_sampled():
    wl = workloads.workload("fan512_cubic")
    g, og = _grid(wl.n, wl.degree, wl.h)
    lines = device_lines(wl.geometry, DEV)
    th, yy = oracle_lines(wl.geometry)
    sino = sp.spline_project_fwd(g, torch.from_numpy(wl.coef).to(DEV), lines).cpu().numpy()
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(th.size, 300, replace=False))
    ref = oracle.forward(og, wl.coef, th[idx], yy[idx])
    assert rel_l2(sino[idx], ref) < TOL
    # adjoint: backproject the projection, check sampled nodes one by one
    p = sino.astype(np.float32)
    back = sp.spline_project_adj(g, torch.from_numpy(p).to(DEV), lines).cpu().numpy().ravel()
    pix = np.sort(rng.choice(wl.n * wl.n, 40, replace=False))
    ref_b = oracle.adjoint_pixels(og, p.astype(np.float64), th, yy, pix)
    assert rel_l2(back[pix], ref_b) < TOL


# ------------------------------------------------------------------ edge cases
def test_degree0_axis_ties_midpoint():
    # theta = 0 and pi/2 with offsets on cell edges: the line runs along cell
    # boundaries and each neighbour takes half (midpoint convention).
    g, og = _grid(16, 0)
    view = np.array([0.0, math.pi / 2, 0.7], dtype=np.float32)
    geo = workloads.Geometry("parallel", view_angle=view, n_det=33, det0=-8.0, ddet=0.5)
    coef = np.random.default_rng(2).uniform(-1, 1, (16, 16)).astype(np.float32)
    lines = device_lines(geo, DEV)
    th, yy = oracle_lines(geo)
    sino = sp.spline_project_fwd(g, torch.from_numpy(coef).to(DEV), lines).cpu().numpy()
    ref = oracle.forward(og, coef, th, yy, brute=True)
    np.testing.assert_allclose(sino, ref, rtol=1e-5, atol=1e-5)
    # the visited set on the exactly axis-aligned view (theta = fl(pi/2) is
    # 4e-8 off the axis and puts pairs within 1e-15 of the open support
    # boundary, where phi = 0 and either decision is exact to rounding)
    counts = sp.spline_visited(g, lines).cpu().numpy()[:33]
    rc, _ = oracle.visited(og, th[:33], yy[:33], brute=True)
    assert np.array_equal(counts.astype(np.int64), rc)


@pytest.mark.parametrize("kind", ["parallel", "fan"])
def test_degree0_on_strip_kernels(kind):
    # degree 0 runs on the general kernels by default; set to the strip
    # kernels (as the autotuner may) it keeps the parity bar, including the
    # views exactly along an axis (midpoint rule, handled line by line)
    g, og = _grid(40, 0)
    if kind == "parallel":
        view = np.array([0.0, 0.3, math.pi / 2, 1.9, 2.6], dtype=np.float32)
        geo = workloads.Geometry("parallel", view_angle=view, n_det=70, det0=-34.5, ddet=1.0)
    else:
        geo = _small_geometry("fan", 0, 21)
    coef = np.random.default_rng(5).uniform(-1, 1, (40, 40)).astype(np.float32)
    lines = device_lines(geo, DEV)
    th, yy = oracle_lines(geo)
    plan = sp.Plan(g, lines)
    plan.set_paths(1, 1)
    sino = plan.fwd(torch.from_numpy(coef).to(DEV))
    ref = oracle.forward(og, coef, th, yy)
    assert rel_l2(sino.cpu().numpy(), ref) < TOL
    p = np.random.default_rng(6).uniform(-1, 1, th.size).astype(np.float32)
    back = plan.adj(torch.from_numpy(p).to(DEV)).cpu().numpy()
    assert rel_l2(back, oracle.adjoint(og, p.astype(np.float64), th, yy)) < TOL
    plan.set_paths(2, 2)
    assert float((plan.fwd(torch.from_numpy(coef).to(DEV)) - sino).norm() / sino.norm()) < 1e-6


def test_empty_and_missing_lines():
    g, og = _grid(20, 3)
    empty = sp.Lines.theta_y(torch.zeros(0, device=DEV), torch.zeros(0, device=DEV))
    coef = torch.ones(20, 20, device=DEV)
    assert sp.spline_project_fwd(g, coef, empty).numel() == 0
    assert float(sp.spline_project_adj(g, torch.zeros(0, device=DEV), empty).abs().sum()) == 0.0
    far = sp.Lines.theta_y(torch.tensor([0.3, 1.2], device=DEV), torch.tensor([100.0, -60.0], device=DEV))
    assert float(sp.spline_project_fwd(g, coef, far).abs().max()) == 0.0


@pytest.mark.parametrize("nx,ny,kind", [(2048, 2048, "fan"), (4096, 96, "parallel")])
def test_large_grids_sampled(nx, ny, kind):
    # grids beyond the benchmark's: index arithmetic over 4 M nodes, long
    # major-axis rows, and a flat grid whose lines leave it after a few rows
    n = 3
    g, og = sp.Grid(nx, ny, n, 1.0), oracle.Grid(nx, ny, n, 1.0)
    if kind == "fan":
        geo = workloads.Geometry("fan", view_angle=np.linspace(0.05, 2 * math.pi, 12, endpoint=False).astype(np.float32),
                                 n_det=3072, det0=-1535.5, ddet=1.0, dso=4000.0, dod=2000.0)
    else:
        geo = workloads.Geometry("parallel", view_angle=np.array([0.0, 0.2, 0.9, 1.5707964, 2.5], dtype=np.float32),
                                 n_det=4200, det0=-2099.5, ddet=1.0)
    rng = np.random.default_rng(nx + ny)
    coef = rng.uniform(-1, 1, (ny, nx)).astype(np.float32)
    lines = device_lines(geo, DEV)
    th, yy = oracle_lines(geo)
    plan = sp.Plan(g, lines)
    sino = plan.fwd(torch.from_numpy(coef).to(DEV)).cpu().numpy()
    idx = np.sort(rng.choice(th.size, 200, replace=False))
    assert rel_l2(sino[idx], oracle.forward(og, coef, th[idx], yy[idx])) < TOL
    p = rng.uniform(-1, 1, th.size).astype(np.float32)
    back = plan.adj(torch.from_numpy(p).to(DEV)).cpu().numpy().ravel()
    pix = np.sort(rng.choice(nx * ny, 16, replace=False))
    assert rel_l2(back[pix], oracle.adjoint_pixels(og, p.astype(np.float64), th, yy, pix)) < TOL


def test_tiny_and_rectangular_grids():
    for (nx, ny, n) in [(1, 1, 3), (1, 7, 2), (9, 1, 1), (3, 40, 3)]:
        g = sp.Grid(nx, ny, n, 1.3, 0.2, -0.4)
        og = oracle.Grid(nx, ny, n, 1.3, 0.2, -0.4)
        rng = np.random.default_rng(nx * 100 + ny)
        th = rng.uniform(0, 2 * math.pi, 400).astype(np.float32)
        yy = rng.uniform(-0.8 * max(nx, ny), 0.8 * max(nx, ny), 400).astype(np.float32)
        coef = rng.uniform(-1, 1, (ny, nx)).astype(np.float32)
        lines = sp.Lines.theta_y(torch.from_numpy(th).to(DEV), torch.from_numpy(yy).to(DEV))
        got = sp.spline_project_fwd(g, torch.from_numpy(coef).to(DEV), lines).cpu().numpy()
        ref = oracle.forward(og, coef, th, yy, brute=True)
        assert rel_l2(got, ref) < TOL
        back = sp.spline_project_adj(g, torch.from_numpy(got).to(DEV), lines).cpu().numpy()
        assert rel_l2(back, oracle.adjoint(og, got.astype(np.float64), th, yy)) < TOL


def test_lines_expand_matches_oracle():
    for geo in (_small_geometry("fan", 30, 1), _small_geometry("parallel", 30, 2),
                _small_geometry("points", 30, 3)):
        lines = device_lines(geo, DEV)
        th, yy = sp.spline_lines_expand(lines)
        rth, ryy = oracle_lines(geo)
        # same line: directions agree up to orientation and offsets accordingly
        d = np.angle(np.exp(1j * (th.cpu().numpy().astype(np.float64) - rth)))
        assert np.abs(d).max() < 1e-6
        assert np.abs(yy.cpu().numpy() - ryy).max() < 1e-4


def test_invalid_arguments_rejected():
    coef = torch.zeros(4, 4, device=DEV)
    lines = sp.Lines.theta_y(torch.zeros(3, device=DEV), torch.zeros(3, device=DEV))
    with pytest.raises(sp.SplineError):
        sp.spline_project_fwd(sp.Grid(4, 4, 5), coef, lines)
    with pytest.raises(sp.SplineError):
        sp.spline_project_fwd(sp.Grid(4, 4, 1, h=0.0), coef, lines)


@pytest.mark.parametrize("name", ["fan512_cubic", "fan256_cubic", "parallel64_linear", "parallel256_cubic"])
def test_strip_windows_cover_every_run(name):
    # The forward stages, per group of neighbouring lines, one window of
    # coefficients per row; every run of nonzero nodes should fall inside it.
    wl = workloads.workload(name)
    g, _ = _grid(wl.n, wl.degree, wl.h)
    lines = device_lines(wl.geometry, DEV)
    plan = sp.Plan(g, lines)
    plan.fwd(torch.from_numpy(wl.coef).to(DEV))
    assert plan.slow_rows() == 0
    plan.close()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_diagonal_and_axis_lines_through_nodes(n):
    # directions where sin and cos round to the same float (or one vanishes),
    # on lines through nodes: rows step by the exact |kappa|, the tables use
    # the float a
    N = 24
    g, og = _grid(N, n)
    base = [0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, math.pi, 5 * math.pi / 4]
    th = np.repeat(np.array(base, dtype=np.float32), 33)
    y = np.tile(np.linspace(-16.0, 16.0, 33), len(base)).astype(np.float32)
    coef = workloads.ellipse_phantom(N, 6, 43, radius=8.0, axes=(2.0, 7.0))
    lines = sp.Lines.theta_y(torch.from_numpy(th).to(DEV), torch.from_numpy(y).to(DEV))
    sino = sp.spline_project_fwd(g, torch.from_numpy(coef).to(DEV), lines).cpu().numpy()
    assert rel_l2(sino, oracle.forward(og, coef, th.astype(np.float64), y.astype(np.float64))) < TOL


@pytest.mark.parametrize("records", [False, True])
def test_adjoint_float_strips_for_extreme_and_nonfinite_values(records):
    # A chunk whose sinogram values are too large or too small for its
    # fixed-point scale, or not finite, accumulates its strip in FP32 (an
    # out-of-line copy of the strip adjoint): views of values ~1e25 and
    # ~1e-25 beside ordinary ones, against the warp-per-line adjoint and the
    # oracle; a NaN reaches exactly the nodes its line touches.
    W = workloads.crop_workload(workloads.workload("fan512_cubic"), 64, seed=13)
    g, og = _grid(W.n, W.degree, W.h)
    lines = device_lines(W.geometry, DEV)
    nd = W.geometry.n_det
    rng = np.random.default_rng(8)
    p = rng.uniform(0.5, 1.5, lines.m)
    p[:nd] *= 1e25
    p[nd:2 * nd] *= 1e-25
    p = p.astype(np.float32)
    plan = sp.Plan(g, lines, prepare=True, records=records)
    back = plan.adj(torch.from_numpy(p).to(DEV)).clone()
    plan.set_paths(0, 2)
    ref = plan.adj(torch.from_numpy(p).to(DEV))
    torch.cuda.synchronize()
    assert float((back - ref).double().norm() / ref.double().norm()) < 1e-6
    th, yy = oracle_lines(W.geometry)
    assert rel_l2(back.cpu().numpy(), oracle.adjoint(og, p.astype(np.float64), th, yy)) < TOL
    # the second view alone (tiny values) against the oracle, to its own scale
    q = np.zeros_like(p)
    q[nd:2 * nd] = p[nd:2 * nd]
    plan.set_paths(0, 0)
    small = plan.adj(torch.from_numpy(q).to(DEV)).cpu().numpy()
    assert rel_l2(small, oracle.adjoint(og, q.astype(np.float64), th, yy)) < TOL
    # a NaN reaches every node the line's footprint covers, and nothing
    # farther than the neighbours of those (the row's candidate slots at the
    # ends of its run, where the footprint is 0, get NaN * 0 too)
    r = np.ones_like(p)
    r[3 * nd + 100] = np.nan
    got = np.isnan(plan.adj(torch.from_numpy(r).to(DEV)).cpu().numpy())
    mask = np.zeros(lines.m)
    mask[3 * nd + 100] = 1.0
    touched = oracle.adjoint(og, mask, th, yy) != 0.0
    assert touched.any() and np.all(got[touched])
    near = np.pad(touched, 1)
    near = np.logical_or.reduce([near[1 + di:near.shape[0] - 1 + di, 1 + dj:near.shape[1] - 1 + dj]
                                 for di in (-1, 0, 1) for dj in (-1, 0, 1)])
    assert not np.any(got & ~near)
    plan.close()
