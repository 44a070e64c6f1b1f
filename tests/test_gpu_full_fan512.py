"""Whole-sinogram parity at the benchmark's own size and launch configuration:
512 x 512 cubic B-splines, fan beam of 720 views x 768 bins (dso 1000,
dod 500), 30-ellipse phantom, through a prepared plan as bench.py runs it.

Forward: every one of the 552,960 lines against the FP64 oracle (about 40 s
on 16 host cores), relative L2 over the whole sinogram <= 1e-5.
Adjoint: the backprojection of that sinogram on every node of the grid's
border (corners included) and 600 random interior nodes, each computed by
the oracle node by node over all lines, relative L2 <= 1e-5."""
import numpy as np
import pytest

import oracle
import workloads
from _geom import device_lines, oracle_lines, rel_l2

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def fan512():
    oracle.build()
    wl = workloads.workload("fan512_cubic")
    dev = torch.device("cuda")
    grid = sp.Grid(wl.n, wl.n, wl.degree, wl.h)
    lines = device_lines(wl.geometry, dev)
    plan = sp.Plan(grid, lines, prepare=True)
    coef = torch.from_numpy(wl.coef).to(dev)
    sino = plan.fwd(coef)
    back = plan.adj(sino)
    torch.cuda.synchronize()
    th, yy = oracle_lines(wl.geometry)
    og = oracle.Grid(wl.n, wl.n, wl.degree, wl.h)
    return wl, og, th, yy, sino.cpu().numpy(), back.cpu().numpy().ravel()


def test_fan512_cubic_whole_sinogram(fan512):
    wl, og, th, yy, sino, _ = fan512
    assert th.size == 552960 and np.isfinite(sino).all()
    ref = oracle.forward(og, wl.coef, th, yy)
    assert rel_l2(sino, ref) < TOL
    # no view far off either: the worst view's relative L2 stays small too
    per_view = np.linalg.norm((sino - ref).reshape(720, 768), axis=1) / \
        np.maximum(np.linalg.norm(ref.reshape(720, 768), axis=1), 1e-30)
    assert per_view.max() < 1e-4


def test_fan512_cubic_backprojection_border_and_interior_nodes(fan512):
    wl, og, th, yy, sino, back = fan512
    n = wl.n
    idx = np.arange(n)
    border = np.unique(np.concatenate([idx, (n - 1) * n + idx, idx * n, idx * n + n - 1]))
    rng = np.random.default_rng(2024)
    inner = rng.choice(np.setdiff1d(np.arange(n * n), border), 600, replace=False)
    pix = np.sort(np.concatenate([border, inner]))
    assert pix.size >= 2000 and {0, n - 1, (n - 1) * n, n * n - 1} <= set(pix.tolist())
    ref = oracle.adjoint_pixels(og, sino.astype(np.float64), th, yy, pix)
    assert rel_l2(back[pix], ref) < TOL
    assert rel_l2(back[border], ref[np.isin(pix, border)]) < TOL
