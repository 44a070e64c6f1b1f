"""The uneven 64-instance batch at full size, in the launch configuration the
benchmark times (one CUDA graph per direction, persistent queue kernel for
the strip-eligible instances, autotuned paths), against the FP64 oracle on
sampled outputs: 150 lines of every instance's projection and 6 nodes of the
backprojection of every eighth instance, each within relative L2 1e-5."""
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
COUNT = 64


@pytest.fixture(scope="module")
def full_batch():
    ws = [workloads.batch_instance(i, 1.0) for i in range(COUNT)]
    grids = [sp.Grid(w.n, w.n, w.degree, w.h) for w in ws]
    lines = [device_lines(w.geometry, DEV) for w in ws]
    coefs = [torch.from_numpy(w.coef).to(DEV) for w in ws]
    batch = sp.Batch(grids, lines)
    sinos = batch.fwd(coefs)
    backs = batch.adj(sinos)
    paths = batch.autotune(coefs, sinos)
    sinos = batch.fwd(coefs, sinos)
    backs = batch.adj(sinos, backs)
    torch.cuda.synchronize()
    yield ws, grids, lines, batch, paths, [s.cpu().numpy() for s in sinos], [b.cpu().numpy() for b in backs]
    batch.close()


def test_full_batch_ran_through_queue(full_batch):
    ws, grids, lines, batch, paths, sinos, backs = full_batch
    # the queue kernels carry every instance on the strip kernels (one
    # persistent launch per degree and direction), any line-list kind
    n_fwd = sum(1 for (f, _) in paths if f == 1)
    n_adj = sum(1 for (_, a) in paths if a == 1)
    assert batch.queued(False) == n_fwd and batch.queued(True) == n_adj
    assert n_adj > 0


def test_full_batch_forward_sampled(full_batch):
    ws, grids, lines, batch, paths, sinos, backs = full_batch
    for k, w in enumerate(ws):
        og = oracle.Grid(w.n, w.n, w.degree, w.h)
        th, yy = oracle_lines(w.geometry)
        idx = np.sort(np.random.default_rng(500 + k).choice(th.size, 150, replace=False))
        ref = oracle.forward(og, w.coef, th[idx], yy[idx])
        assert rel_l2(sinos[k][idx], ref) < TOL, (k, w.n, w.degree, w.geometry.kind)


def test_full_batch_adjoint_sampled(full_batch):
    ws, grids, lines, batch, paths, sinos, backs = full_batch
    for k in range(0, COUNT, 8):
        w = ws[k]
        og = oracle.Grid(w.n, w.n, w.degree, w.h)
        th, yy = oracle_lines(w.geometry)
        # nodes near the centre, where every view contributes
        rng = np.random.default_rng(900 + k)
        c = w.n // 2
        ii = rng.integers(c - w.n // 4, c + w.n // 4, 6)
        jj = rng.integers(c - w.n // 4, c + w.n // 4, 6)
        pix = jj * w.n + ii
        ref = oracle.adjoint_pixels(og, sinos[k].astype(np.float64), th, yy, pix)
        assert rel_l2(backs[k].ravel()[pix], ref) < TOL, (k, w.n, w.degree, w.geometry.kind)
