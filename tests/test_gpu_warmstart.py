"""The trained warm start (paper_2503_20907_gb300/weights): the network run
through this library's kernels against the FP64 oracle layers with the same
BF16 rounding between layers, and what it gains over plain CGLS on held-out
samples, measured and printed: a smaller starting normal-equation residual,
and iteration counts to relative residuals of 1e-3 and 1e-4 that stay within
a couple of iterations of cold CGLS (the last decades are spent on
components of small eigenvalue that the network does not predict)."""
import numpy as np
import pytest

from oracle.conv import conv3x3

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def trained():
    from paper_2503_20907_gb300 import warmstart as ws
    net, meta = ws.load_net(ws.DEFAULT_WEIGHTS, DEV)
    return ws, net, meta


def test_network_forward_matches_oracle_layers(trained):
    ws, net, meta = trained
    rng = np.random.default_rng(0)
    z = torch.from_numpy(rng.standard_normal((1, 48, 80)).astype(np.float32)).to(DEV)
    with torch.no_grad():
        got = net(z).cpu().numpy()[0]
    # reference: FP64 layers, activations rounded to BF16 after each layer as the kernels store them
    x = z.to(torch.bfloat16).float().cpu().numpy()[..., None].astype(np.float64)
    for k, (cin, cout, relu, dil) in enumerate(ws.LAYERS):
        w = net.w[k].detach().to(torch.bfloat16).float().cpu().numpy()
        y = conv3x3(x, w, net.b[k].detach().cpu().numpy(), d=dil)
        if relu:
            y = np.maximum(y, 0.0)
        x = y if cout == 1 else torch.from_numpy(y).to(torch.bfloat16).double().numpy()
    ref = z.cpu().numpy()[0] + x[0, :, :, 0]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-3


def test_warm_start_gain_on_held_out_samples(trained):
    ws, net, meta = trained
    grid, lines = ws.geometry(DEV)
    plan = sp.Plan(grid, lines)
    n = 24
    z, c, b, _ = ws.make_samples(plan, [2_000_000 + i for i in range(n)], DEV, meta["alpha"])
    rel0, kc, kw, kc3, kw3 = [], [], [], [], []
    for k in range(n):
        _, gc = plan.cgls(b[k], 800)
        gc = gc.cpu().numpy()
        with torch.no_grad():
            x0 = net(z[k:k + 1])[0]
        _, gz = plan.cgls(b[k], 0, x0=z[k])
        _, gw = plan.cgls(b[k], 800, x0=x0)
        gw = gw.cpu().numpy()
        rel0.append((np.sqrt(gw[0] / gc[0]), np.sqrt(float(gz[0]) / gc[0])))
        kc.append(ws.iterations_to(gc, gc[0], 1e-4))
        kw.append(ws.iterations_to(gw, gc[0], 1e-4))
        kc3.append(ws.iterations_to(gc, gc[0], 1e-3))
        kw3.append(ws.iterations_to(gw, gc[0], 1e-3))
    # every sample reaches 1e-3; a rare one stalls above 1e-4 within the 800
    # FP32 iterations (1 of 256 cold in the benchmark's run): compare the
    # samples that reach it both ways
    assert all(x is not None for x in kc3 + kw3)
    both = [i for i in range(n) if kc[i] is not None and kw[i] is not None]
    assert len(both) >= n - 2
    kc4, kw4 = [kc[i] for i in both], [kw[i] for i in both]
    print(f"\nwarm start on {n} held-out samples: starting residual {np.median([a for a, _ in rel0]):.3f} "
          f"(cold 1, z alone {np.median([b_ for _, b_ in rel0]):.3f}); iterations to 1e-3 "
          f"{np.median(kw3):.1f} warm vs {np.median(kc3):.1f} cold (mean {np.mean(kw3):.2f} vs {np.mean(kc3):.2f}); "
          f"to 1e-4 ({len(both)} samples) {np.median(kw4):.1f} vs {np.median(kc4):.1f}")
    # the network's start is closer than 0, and (median) than its input z, in
    # the normal-equation residual (it is trained on the residual left after
    # 12 CGLS steps, not on the starting one)
    assert np.median([rw for rw, _ in rel0]) < 0.5
    assert np.median([rw for rw, _ in rel0]) < np.median([rz for _, rz in rel0])
    # the iteration counts: within a couple of iterations of cold CGLS at
    # both tolerances (the gain of the lower starting residual is about one
    # iteration, the size of the sample-to-sample spread of a 24-sample
    # median; the benchmark reports it on 256 samples)
    assert abs(np.mean(kw3) - np.mean(kc3)) <= 2
    assert abs(np.median(kw4) - np.median(kc4)) <= 4
    # the solver with fallback returns a solution within the tolerance either way
    x, iters, warm = ws.solve(plan, b[0], net, meta["alpha"], tol=1e-4)
    s = plan.adj(plan.fwd(x) - b[0])
    s0 = plan.adj(b[0])
    assert float(s.norm() / s0.norm()) < 5e-4   # recursive CGLS residual vs the one recomputed in FP32
