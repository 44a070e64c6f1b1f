"""Row records kept by a plan: spline_plan_prepare stores every line's sorted
row records once, and the plan's projections replay them instead of
traversing the rows again.  The replay must give what the one-shot entry
points (which always traverse) give: the forward bit for bit (same phase B
arithmetic in the same order), the adjoint to rounding (its image additions
from different blocks come in any order), and both against the oracle."""
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


def _rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / max(float(b.norm()), 1e-300))


CASES = [   # (workload cropped to n x n, degree, basis: 0 B-spline, 1 three-direction box-spline)
    ("fan512_cubic", 128, 3, 0),
    ("fan512_cubic", 96, 1, 0),
    ("fan512_cubic", 72, 1, 1),
    ("parallel256_cubic", 128, 2, 0),
    ("parallel256_cubic", 80, 3, 0),
]


@pytest.mark.parametrize("base,n,degree,basis", CASES)
def test_plan_replay_matches_one_shot_and_oracle(base, n, degree, basis):
    W = workloads.crop_workload(workloads.workload(base), n, degree=degree, seed=21)
    grid = sp.Grid(W.n, W.n, W.degree, W.h, basis=basis)
    lines = device_lines(W.geometry, DEV)
    coef = torch.from_numpy(W.coef).to(DEV)
    plan = sp.Plan(grid, lines, prepare=True, records=True)
    assert plan.record_bytes() > 0
    got = plan.fwd(coef)
    ref = sp.spline_project_fwd(grid, coef, lines)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    # adjoint of a sinogram with zero lines (skipped by the replay, not by the groups)
    p = torch.randn(lines.m, device=DEV, generator=torch.Generator(DEV).manual_seed(3))
    p[::3] = 0.0
    back = plan.adj(p)
    back_ref = sp.spline_project_adj(grid, p, lines)
    assert _rel(back, back_ref) < 1e-6
    th, yy = oracle_lines(W.geometry)
    og = oracle.Grid(W.n, W.n, W.degree, W.h, basis=basis)
    assert rel_l2(got.cpu().numpy(), oracle.forward(og, W.coef, th, yy)) < 1e-5
    assert rel_l2(back.cpu().numpy(), oracle.adjoint(og, p.cpu().numpy().astype(np.float64), th, yy)) < 1e-5
    plan.close()


def test_plan_records_follow_a_new_prepare():
    # new view angles in the same device buffer: prepare rewrites the records
    W = workloads.crop_workload(workloads.workload("fan512_cubic"), 64, seed=8)
    geo = W.geometry
    view = torch.from_numpy(geo.view_angle).to(DEV)
    lines = sp.Lines.fan(view, geo.dso, geo.dod, geo.n_det, geo.det0, geo.ddet)
    grid = sp.Grid(W.n, W.n, W.degree, W.h)
    coef = torch.from_numpy(W.coef).to(DEV)
    plan = sp.Plan(grid, lines, prepare=True, records=True)
    assert plan.record_bytes() > 0
    first = plan.fwd(coef).clone()
    view.add_(0.37)
    plan.prepare()
    again = plan.fwd(coef)
    ref = sp.spline_project_fwd(grid, coef, lines)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)
    assert not torch.equal(again, first)
    plan.close()


def test_plan_replay_in_cgls_matches_oracle_first_iterate():
    # CGLS runs its projections through the plan, i.e. on the kept records
    W = workloads.crop_workload(workloads.workload("fan512_cubic"), 48, seed=4)
    grid = sp.Grid(W.n, W.n, W.degree, W.h)
    lines = device_lines(W.geometry, DEV)
    plan = sp.Plan(grid, lines, prepare=True, records=True)
    assert plan.record_bytes() > 0
    th, yy = oracle_lines(W.geometry)
    og = oracle.Grid(W.n, W.n, W.degree, W.h)
    b = oracle.forward(og, W.coef.astype(np.float64), th, yy)
    x, _ = plan.cgls(torch.from_numpy(b.astype(np.float32)).to(DEV), 1)
    s = oracle.adjoint(og, b, th, yy)
    q = oracle.forward(og, s, th, yy)
    x1 = (s * s).sum() / (q * q).sum() * s
    assert rel_l2(x.cpu().numpy(), x1) < 2e-5
    plan.close()


def test_records_only_where_they_apply_and_can_be_dropped():
    W = workloads.crop_workload(workloads.workload("fan512_cubic"), 32, degree=0, seed=2)
    plan = sp.Plan(sp.Grid(W.n, W.n, 0, W.h), device_lines(W.geometry, DEV), prepare=True)
    assert plan.record_bytes() == 0
    with pytest.raises(sp.SplineError):
        plan.set_records(True)
    plan.close()
    W = workloads.crop_workload(workloads.workload("fan512_cubic"), 32, seed=2)
    grid, lines = sp.Grid(W.n, W.n, W.degree, W.h), device_lines(W.geometry, DEV)
    plan = sp.Plan(grid, lines, prepare=True)
    assert plan.record_bytes() == 0          # new plans keep none
    coef = torch.from_numpy(W.coef).to(DEV)
    a = plan.fwd(coef).clone()
    plan.set_records(True)
    assert plan.record_bytes() > 0
    b = plan.fwd(coef).clone()
    plan.set_records(False)
    assert plan.record_bytes() == 0
    c = plan.fwd(coef)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)
    plan.close()
