"""CGLS at the full size of the reconstruction workload (512 x 512 cubic,
fan 720 x 768, transmission data with Poisson noise at 1e4 photons, 100
iterations), in the launch configuration the benchmark times.  The FP64
oracle cannot run the whole solve in seconds, so the checks are the ones
that hold at any size: the first iterate is a multiple of A^T b (checked on
sampled nodes against the oracle's backprojection), the data misfit of CGLS
never grows, and the normal-equation residual falls by four decades."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _geom import device_lines, oracle_lines, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full_cg():
    import paper_2503_20907_gb300 as sp
    oracle.build()
    wl = workloads.workload("fan512_cubic")
    dev = torch.device("cuda")
    plan = sp.Plan(sp.Grid(wl.n, wl.n, wl.degree, wl.h), device_lines(wl.geometry, dev))
    coef = torch.from_numpy(wl.coef).to(dev)
    b_np, _ = workloads.transmission_data(plan.fwd(coef).cpu().numpy(), seed=3)
    b = torch.from_numpy(b_np.astype(np.float32)).to(dev)
    return wl, plan, b


def test_first_iterate_is_scaled_backprojection(full_cg):
    wl, plan, b = full_cg
    x1, _ = plan.cgls(b, 1)
    th, yy = oracle_lines(wl.geometry)
    og = oracle.Grid(wl.n, wl.n, wl.degree, wl.h)
    rng = np.random.default_rng(31)
    c = wl.n // 2
    ii = rng.integers(c - 160, c + 160, 24)
    jj = rng.integers(c - 160, c + 160, 24)
    pix = jj * wl.n + ii
    s0 = oracle.adjoint_pixels(og, b.cpu().numpy().astype(np.float64), th, yy, pix)
    got = x1.cpu().numpy().ravel()[pix].astype(np.float64)
    alpha = float(got @ s0 / (s0 @ s0))
    assert alpha > 0
    assert rel_l2(got, alpha * s0) < 1e-5


def test_misfit_never_grows_and_residual_falls(full_cg):
    wl, plan, b = full_cg
    mis = []
    for k in (10, 25, 50, 100):
        x, gam = plan.cgls(b, k)
        mis.append(float((plan.fwd(x) - b).double().norm()))
    assert all(m2 <= m1 * (1 + 1e-6) for m1, m2 in zip(mis, mis[1:])), mis
    g = gam.cpu().numpy()
    assert np.all(np.isfinite(g))
    assert np.sqrt(g[-1] / g[0]) < 5e-4
