"""Batches of uneven instances (one CUDA graph per set of data pointers) and
the autotuner's kernel choice: the batch gives what each instance's own plan
gives, replays and re-records correctly, and every kernel choice keeps the
oracle parity bar (relative L2 <= 1e-5)."""
import numpy as np
import pytest

import oracle
import workloads
from _geom import device_lines, oracle_lines, rel_l2

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _instances():
    ws = [workloads.batch_instance(i, 0.12) for i in range(12)]
    # plus a box-spline fan instance
    base = workloads.crop_workload(workloads.workload("fan512_cubic"), 40)
    return ws, base


@pytest.fixture(scope="module")
def batch_setup():
    ws, box = _instances()
    grids = [sp.Grid(w.n, w.n, w.degree, w.h) for w in ws] + [sp.Grid(box.n, box.n, 1, box.h, basis=sp.BASIS_BOX3)]
    lines = [device_lines(w.geometry, DEV) for w in ws] + [device_lines(box.geometry, DEV)]
    coefs = [torch.from_numpy(w.coef).to(DEV) for w in ws] + [torch.from_numpy(box.coef).to(DEV)]
    batch = sp.Batch(grids, lines)
    plans = [sp.Plan(g, L) for g, L in zip(grids, lines)]
    return ws + [box], grids, lines, coefs, batch, plans


def test_batch_matches_plans_and_replays(batch_setup):
    ws, grids, lines, coefs, batch, plans = batch_setup
    sinos = batch.fwd(coefs)
    torch.cuda.synchronize()
    for s, p, c in zip(sinos, plans, coefs):
        assert torch.equal(s, p.fwd(c))          # same kernels, deterministic forward
    again = batch.fwd(coefs, sinos=[torch.empty_like(s) for s in sinos])   # new pointers: re-recorded
    for a, b in zip(again, sinos):
        assert torch.equal(a, b)
    same = batch.fwd(coefs, sinos=again)        # same pointers: replayed graph
    for a, b in zip(same, sinos):
        assert torch.equal(a, b)
    backs = batch.adj(sinos)
    for bk, p, s in zip(backs, plans, sinos):
        ref = p.adj(s)
        assert float((bk - ref).norm() / ref.norm().clamp_min(1e-30)) < 1e-6
    # the strip-eligible instances ran through the persistent queue kernel
    # (parallel and fan beams, and free lists through their sorted order)
    n_strip = sum(1 for g in grids if g.degree >= 1)
    assert n_strip >= 2
    assert batch.queued(False) == n_strip and batch.queued(True) == n_strip


def test_batch_instances_match_oracle(batch_setup):
    ws, grids, lines, coefs, batch, plans = batch_setup
    sinos = batch.fwd(coefs)
    for k in (0, 2, 7, len(ws) - 1):
        w, g = ws[k], grids[k]
        og = oracle.Grid(w.n, w.n, g.degree, w.h, basis=g.basis)
        th, yy = oracle_lines(w.geometry)
        idx = np.arange(th.size) if th.size <= 3000 else np.random.default_rng(k).choice(th.size, 3000, replace=False)
        ref = oracle.forward(og, w.coef, th[idx], yy[idx])
        assert rel_l2(sinos[k].cpu().numpy()[idx], ref) < 1e-5


def test_autotune_choices_keep_parity(batch_setup):
    ws, grids, lines, coefs, batch, plans = batch_setup
    sinos = [p.fwd(c) for p, c in zip(plans, coefs)]
    paths = batch.autotune(coefs, sinos)
    assert len(paths) == len(ws)
    for (f, a), L, g in zip(paths, lines, grids):
        assert f in (1, 2) and a in (1, 2)
    out = batch.fwd(coefs)
    back = batch.adj(sinos)
    for k in (1, 3, len(ws) - 1):
        w, g = ws[k], grids[k]
        og = oracle.Grid(w.n, w.n, g.degree, w.h, basis=g.basis)
        th, yy = oracle_lines(w.geometry)
        assert rel_l2(out[k].cpu().numpy(), oracle.forward(og, w.coef, th, yy)) < 1e-5
        assert rel_l2(back[k].cpu().numpy(), oracle.adjoint(og, sinos[k].cpu().numpy(), th, yy)) < 1e-5


def test_general_and_strip_kernels_agree(batch_setup):
    ws, grids, lines, coefs, batch, plans = batch_setup
    for p, c, L, g in zip(plans, coefs, lines, grids):
        p.set_paths(1, 1)
        s1 = p.fwd(c)
        b1 = p.adj(s1)
        p.set_paths(2, 2)
        s2 = p.fwd(c)
        b2 = p.adj(s1)
        p.set_paths(0, 0)
        assert float((s1 - s2).norm() / s2.norm()) < 1e-6
        assert float((b1 - b2).norm() / b2.norm()) < 1e-6


def _mixed_instances():
    """Edge cases of the queue: a chunk of fewer than 32 lines, one view, a
    rectangular grid whose rows are not whole 16-byte chunks, degree 0 (off
    the queue by default), a free line list (on the queue in its sorted
    order), a grid smaller than the support."""
    rng = np.random.default_rng(77)
    specs = []
    # (grid, lines-maker)
    specs.append((sp.Grid(37, 23, 3, 1.0), lambda: sp.Lines.fan(
        torch.tensor([0.3], dtype=torch.float32, device=DEV), 90.0, 45.0, 5, -2.0, 1.0)))
    specs.append((sp.Grid(50, 30, 2, 0.9, 1.5, -0.5), lambda: sp.Lines.parallel(
        torch.from_numpy(np.sort(rng.uniform(0, np.pi, 13)).astype(np.float32)).to(DEV), 71, -35.0, 1.0)))
    specs.append((sp.Grid(3, 3, 1, 1.0), lambda: sp.Lines.parallel(
        torch.tensor([0.0, 0.7, 1.5707964], dtype=torch.float32, device=DEV), 9, -4.0, 1.0)))
    specs.append((sp.Grid(40, 40, 0, 1.0), lambda: sp.Lines.parallel(
        torch.tensor([0.0, 0.4, 1.5707964, 2.2, 3.1415927], dtype=torch.float32, device=DEV), 60, -30.0, 1.0)))
    src, dst = workloads.random_lines_circle(700, 30.0, 5)
    specs.append((sp.Grid(40, 40, 3, 1.0), lambda: sp.Lines.points(
        torch.from_numpy(src).to(DEV), torch.from_numpy(dst).to(DEV))))
    grids = [g for g, _ in specs]
    lines = [mk() for _, mk in specs]
    return grids, lines


def test_batch_queue_edge_cases():
    grids, lines = _mixed_instances()
    batch = sp.Batch(grids, lines)
    plans = [sp.Plan(g, L) for g, L in zip(grids, lines)]
    gen = torch.Generator(device="cpu").manual_seed(11)
    coefs = [torch.rand(g.ny, g.nx, generator=gen).to(DEV) for g in grids]
    sinos = batch.fwd(coefs)
    backs = batch.adj(sinos)
    assert batch.queued(False) == 4 and batch.queued(True) == 4
    for s, b, p, c, sn in zip(sinos, backs, plans, coefs, sinos):
        assert torch.equal(s, p.fwd(c))
        ref = p.adj(sn)
        assert float((b - ref).norm() / ref.norm().clamp_min(1e-30)) < 1e-6
    # degree 0 (the general kernels unless tuned or set otherwise) beside the
    # free list: one queued, same results
    b2 = sp.Batch(grids[3:], lines[3:])
    s2 = b2.fwd(coefs[3:])
    assert b2.queued(False) == 1
    for s, p, c in zip(s2, plans[3:], coefs[3:]):
        assert torch.equal(s, p.fwd(c))
    # one queued instance alone
    b3 = sp.Batch(grids[:1], lines[:1])
    s3 = b3.fwd(coefs[:1])
    k3 = b3.adj(s3)
    assert b3.queued(False) == 1 and b3.queued(True) == 1
    assert torch.equal(s3[0], plans[0].fwd(coefs[0]))
    ref = plans[0].adj(s3[0])
    assert float((k3[0] - ref).norm() / ref.norm().clamp_min(1e-30)) < 1e-6
    for b_ in (batch, b2, b3):
        b_.close()


def test_batch_invalid():
    with pytest.raises(sp.SplineError):
        sp.Batch([sp.Grid(8, 8, 5)], [sp.Lines.theta_y(torch.zeros(3, device=DEV), torch.zeros(3, device=DEV))])


def test_batch_defers_chunks_that_need_float_strips():
    # sinogram values too large for a chunk's fixed-point scale, and a NaN:
    # the queue kernel defers those chunks to its float launch; the results
    # are the instances' own adjoints
    grids, lines = _mixed_instances()
    keep = [0, 1, 4]
    grids, lines = [grids[k] for k in keep], [lines[k] for k in keep]
    batch = sp.Batch(grids, lines)
    plans = [sp.Plan(g, L) for g, L in zip(grids, lines)]
    gen = torch.Generator(device="cpu").manual_seed(12)
    sinos = [torch.rand(L.m, generator=gen).to(DEV) + 0.5 for L in lines]
    sinos[1][:71] *= 1e25
    sinos[2][:40] *= 1e-25
    backs = batch.adj(sinos)
    assert batch.queued(True) == 3
    for b, p, s in zip(backs, plans, sinos):
        ref = p.adj(s)
        assert float((b - ref).double().norm() / ref.double().norm()) < 1e-6
    nan = [s.clone() for s in sinos]
    nan[0][2] = float("nan")
    backs = batch.adj(nan)
    for b, p, s in zip(backs, plans, nan):
        ref = p.adj(s)
        assert torch.equal(torch.isnan(b), torch.isnan(ref))
        ok = ~torch.isnan(ref)
        assert float((b[ok] - ref[ok]).double().norm() / ref[ok].double().norm()) < 1e-6
    batch.close()
