"""Learned warm start for the CGLS reconstruction (no paper counterpart).

A small CNN maps the scaled backprojection z = alpha A^T b of noisy data b to
an initial guess x_0 = z + f(z) of the spline coefficients; CGLS
(Plan.cgls) then starts from x_0 instead of 0, and plain CGLS from 0 stays
the fallback.  f has six 3x3 convolution layers (1 -> 32, four 32 -> 32,
32 -> 1; taps 1, 2, 4, 8, 16, 1 apart) with ReLU between them, BF16 weights and activations and FP32
accumulation, all in this library's kernels (include/warmstart_conv.h):
the forward of the inner layers on the tensor cores, the gradients on the
CUDA cores.  Training data (phantom, sinogram, backprojection) come from the
library's projector.

    python -m paper_2503_20907_gb300.warmstart train --out weights.pt
    python -m paper_2503_20907_gb300.warmstart eval --weights weights.pt
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import _lib
from ._lib import Grid, Lines, Plan, _check, _stream, load

from pathlib import Path

CH = 32
DEFAULT_WEIGHTS = Path(__file__).resolve().parent / "weights" / "warmstart_parallel256.pt"
# (cin, cout, relu, dilation): 3x3 taps spread 1, 2, 4, 8, 16, 1 apart, a
# receptive field of 65 x 65 nodes (the normal operator A^T A is non-local)
LAYERS = ((1, CH, True, 1), (CH, CH, True, 2), (CH, CH, True, 4), (CH, CH, True, 8), (CH, CH, True, 16),
          (CH, 1, False, 1))


class _Conv3x3(torch.autograd.Function):
    """One layer: y = relu?(conv3x3(x) + bias) with this library's kernels."""

    @staticmethod
    def forward(ctx, x, w, b, cin, cout, relu, dil):
        B, H, W = x.shape[0], x.shape[1], x.shape[2]
        wb = w.detach().to(torch.bfloat16).contiguous()
        if cout == 1:
            y = torch.empty((B, H, W), dtype=torch.float32, device=x.device)
        else:
            y = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device=x.device)
        _check(load().sp_conv3x3_fwd(B, H, W, cin, cout, dil, x.data_ptr(), wb.data_ptr(), b.detach().data_ptr(),
                                     int(relu), y.data_ptr(), _stream(None)))
        ctx.save_for_backward(x, wb, y)
        ctx.meta = (cin, cout, relu, dil)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, wb, y = ctx.saved_tensors
        cin, cout, relu, dil = ctx.meta
        B, H, W = x.shape[0], x.shape[1], x.shape[2]
        g = gy.float()
        if relu:
            g = g * (y > 0)
        g = g.contiguous()
        dx = None
        if ctx.needs_input_grad[0]:
            dxf = torch.empty((B, H, W, cin), dtype=torch.float32, device=x.device)
            _check(load().sp_conv3x3_bwd_data(B, H, W, cin, cout, dil, g.data_ptr(), wb.data_ptr(), None,
                                              dxf.data_ptr(), _stream(None)))
            dx = dxf.to(x.dtype)
        dw = torch.empty((cout, 3, 3, cin), dtype=torch.float32, device=x.device)
        db = torch.empty(cout, dtype=torch.float32, device=x.device)
        _check(load().sp_conv3x3_bwd_weight(B, H, W, cin, cout, dil, x.data_ptr(), g.data_ptr(), dw.data_ptr(),
                                            db.data_ptr(), _stream(None)))
        return dx, dw, db, None, None, None, None


def conv3x3(x, w, b, relu: bool, dil: int = 1):
    """x BF16 [B,H,W,cin], w FP32 master weights [cout,3,3,cin] (used as BF16), b FP32 [cout]."""
    return _Conv3x3.apply(x, w, b, int(w.shape[3]), int(w.shape[0]), bool(relu), int(dil))


class WarmStartNet(torch.nn.Module):
    """x_0 = z + f(z), z [B,H,W] FP32."""

    def __init__(self, seed: int = 0):
        super().__init__()
        g = torch.Generator().manual_seed(seed)
        self.w = torch.nn.ParameterList()
        self.b = torch.nn.ParameterList()
        for k, (cin, cout, _, _) in enumerate(LAYERS):
            std = math.sqrt(2.0 / (9 * cin))
            w = torch.randn((cout, 3, 3, cin), generator=g) * std
            if k == len(LAYERS) - 1:
                w.zero_()           # starts as the identity map x_0 = z
            self.w.append(torch.nn.Parameter(w))
            self.b.append(torch.nn.Parameter(torch.zeros(cout)))

    def forward(self, z):
        x = z.to(torch.bfloat16).unsqueeze(-1).contiguous()
        for k, (_, _, relu, dil) in enumerate(LAYERS):
            x = conv3x3(x, self.w[k], self.b[k], relu, dil)
        return z + x


# ------------------------------------------------------------------ data
def geometry(device):
    """256 x 256 cubic splines; parallel beam, 360 angles in [0, pi), 384 bins -192 + j."""
    grid = Grid(256, 256, 3)
    view = (torch.arange(360, dtype=torch.float64) * (math.pi / 360)).float().to(device)
    return grid, Lines.parallel(view, 384, -192.0, 1.0)


def make_samples(plan: Plan, seeds, device, alpha: float | None = None, peak: float = 3.0, target_iters: int = 0):
    """(z, target, b, alpha) for the given seeds: b the log-transformed noisy
    data of the sample's phantom c (Poisson at the sample's I0, attenuation
    scaled to `peak`), z = alpha A^T b, and the target c (target_iters = 0)
    or the CGLS reconstruction after target_iters iterations from 0.  alpha
    (if None) is fitted as sum <A^T b, c> / sum <A^T b, A^T b>."""
    import workloads
    n = plan.grid.nx
    prm = [workloads.warmstart_params(s, n) for s in seeds]
    c = workloads.ellipse_images_torch([p for p, _ in prm], n, device)
    zs, bs = [], []
    gen = torch.Generator(device=device)
    for k, s in enumerate(seeds):
        gen.manual_seed(int(s))
        ac = plan.fwd(c[k])
        kappa = peak / float(ac.max().clamp_min(1e-12))
        I0 = prm[k][1]
        counts = torch.poisson(I0 * torch.exp(-kappa * ac.double()), generator=gen)
        b = (-torch.log(counts.clamp_min(1.0) / I0) / kappa).float()
        bs.append(b)
        zs.append(plan.adj(b))
    z = torch.stack(zs)
    if alpha is None:
        alpha = float((z.double() * c.double()).sum() / (z.double() * z.double()).sum())
    if target_iters > 0:
        c = torch.stack([plan.cgls(bk, target_iters, history=False)[0] for bk in bs])
    return z * alpha, c, torch.stack(bs), alpha


# ------------------------------------------------------------------ training
def cgls_residual_after(plan: Plan, x0, b, iters: int):
    """||A^T (b - A x_K)||^2 after K = iters CGLS steps from x0 (the CGLS
    recurrences of spline_plan_cgls), differentiable in x0 through the
    projector's autograd functions: A and A^T are linear, the step lengths
    alpha and beta are differentiable functions of the iterates."""
    from .autograd import backproject, project
    r = b - project(x0, plan)
    s = backproject(r, plan)
    p = s
    gamma = (s * s).sum()
    for _ in range(iters):
        q = project(p, plan)
        alpha = gamma / (q * q).sum().clamp_min(1e-30)
        r = r - alpha * q
        s = backproject(r, plan)
        gamma_new = (s * s).sum()
        p = s + (gamma_new / gamma.clamp_min(1e-30)) * p
        gamma = gamma_new
    return gamma


def train(n_train=20000, batch=16, epochs=1, lr=1e-3, device="cuda", log=print, chunk=500, target_iters=0,
          loss_kind="residual", cg_steps=0, init=None):
    """loss_kind 'residual': mean over the batch of ||A^T (b - A x_K)||^2 / ||A^T b||^2
    where x_K is CGLS after cg_steps iterations from x_0 = net(z) (cg_steps = 0:
    x_0 itself), the quantity CGLS is judged by, differentiated through the
    projector's autograd functions (the residual left after K steps weighs the
    components CG resolves slowly, which decide the iterations to a tight
    tolerance); 'mse': ||x_0 - target||^2 against the phantom (target_iters =
    0) or a CGLS iterate.  init: (net, meta) to continue from."""
    from .autograd import backproject, project
    torch.manual_seed(0)
    grid, lines = geometry(device)
    plan = Plan(grid, lines, records=True)   # many projections per prepare
    t0 = time.time()
    if init is not None:
        alpha = init[1]["alpha"]
    else:
        _, _, _, alpha = make_samples(plan, [1_000_000 + i for i in range(64)], device)
    Z, C, Bs = [], [], []
    for s0 in range(0, n_train, chunk):
        z, c, b, _ = make_samples(plan, [1_000_000 + i for i in range(s0, min(n_train, s0 + chunk))], device, alpha,
                                  target_iters=target_iters)
        Z.append(z)
        C.append(c)
        Bs.append(b)
    Z, C, Bs = torch.cat(Z), torch.cat(C), torch.cat(Bs)
    Gn = torch.stack([plan.adj(Bs[k]).double().pow(2).sum() for k in range(n_train)]).float()   # ||A^T b||^2

    def batch_loss(idx):
        x0 = net(Z[idx])
        if loss_kind == "mse":
            return ((x0 - C[idx]) ** 2).mean()
        tot = 0.0
        for j, k in enumerate(idx.tolist()):
            if cg_steps > 0:
                tot = tot + cgls_residual_after(plan, x0[j], Bs[k], cg_steps) / Gn[k]
            else:
                r = backproject(project(x0[j], plan) - Bs[k], plan)
                tot = tot + (r * r).sum() / Gn[k]
        return tot / len(idx)
    log(f"data: {n_train} samples in {time.time() - t0:.1f} s, alpha {alpha:.4e}")
    net = WarmStartNet().to(device)
    if init is not None:
        net.load_state_dict(init[0].state_dict())
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    steps = epochs * (n_train // batch)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps)
    g = torch.Generator(device=device).manual_seed(1)
    t0 = time.time()
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n_train, device=device, generator=g)
        run = 0.0
        for k in range(n_train // batch):
            idx = perm[k * batch:(k + 1) * batch]
            loss = batch_loss(idx)
            opt.zero_grad(set_to_none=True)
            loss.backward()
            opt.step()
            sched.step()
            run += float(loss.detach()) if k % 50 == 0 else 0.0
            step += 1
        log(f"epoch {ep}: mean loss (sampled) {run / max(1, (n_train // batch) // 50):.5f}, {time.time() - t0:.1f} s")
    with torch.no_grad():
        probe = torch.arange(min(256, n_train), device=device)
        fit = float(batch_loss(probe))
        net_id = WarmStartNet().to(device)
        saved, net = net, net_id
        base = float(batch_loss(probe))
        net = saved
    meta = {"alpha": alpha, "n_train": n_train, "batch": batch, "epochs": epochs, "lr": lr, "loss": loss_kind,
            "target": (f"CGLS iterate {target_iters} from 0" if target_iters else "phantom") if loss_kind == "mse"
            else (f"normal-equation residual after {cg_steps} CGLS steps from x_0" if cg_steps
                  else "normal-equation residual"),
            "cg_steps": cg_steps, "continued_from": (init[1].get("target") if init is not None else None),
            "train_loss_identity": base, "train_loss_net": fit, "train_seconds": time.time() - t0,
            "geometry": "256x256 cubic, parallel 360 angles x 384 bins"}
    return net, meta


def save(net, meta, path):
    torch.save({"state": {k: v.detach().cpu() for k, v in net.state_dict().items()}, "meta": meta}, path)


def load_net(path, device="cuda"):
    d = torch.load(path, map_location="cpu", weights_only=False)
    net = WarmStartNet()
    net.load_state_dict(d["state"])
    return net.to(device), d["meta"]


# ------------------------------------------------------------------ solving
def solve(plan: Plan, b, net=None, alpha: float | None = None, tol: float = 1e-4, max_iters: int = 600):
    """CGLS to ||A^T (b - A x)|| < tol ||A^T b||, warm-started by the network
    when one is given; plain CGLS from 0 is the fallback when the warm start
    does not reach the tolerance.  Returns (x, iterations, warm_used)."""
    x_cold, gc = plan.cgls(b, 0)
    g0 = float(gc[0])
    if net is not None:
        with torch.no_grad():
            z = plan.adj(b) * alpha
            x0 = net(z.unsqueeze(0))[0]
        _, gw = plan.cgls(b, max_iters, x0=x0)
        k = iterations_to(gw.cpu().numpy(), g0, tol)
        if k is not None:
            x, _ = plan.cgls(b, k, x0=x0, history=False)
            return x, k, True
    _, gcold = plan.cgls(b, max_iters)
    k = iterations_to(gcold.cpu().numpy(), g0, tol)
    x, _ = plan.cgls(b, k if k is not None else max_iters, history=False)
    return x, k, False


# ------------------------------------------------------------------ evaluation
def iterations_to(gam: np.ndarray, gamma0: float, tol: float) -> int | None:
    r = np.sqrt(np.maximum(gam, 0.0) / gamma0)
    hit = np.nonzero(r < tol)[0]
    return int(hit[0]) if hit.size else None


def evaluate(net, meta, n_test=256, tol=1e-4, max_iters=600, device="cuda", log=print):
    """Cold (x_0 = 0) vs warm (x_0 = net(z)) CGLS on held-out samples:
    iterations and device time to ||A^T(b - A x_k)|| < tol ||A^T b||."""
    grid, lines = geometry(device)
    plan = Plan(grid, lines)
    z, c, b, _ = make_samples(plan, [2_000_000 + i for i in range(n_test)], device, meta["alpha"])
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))  # noqa: E731
    rows, loose, start = [], [], []
    plan.cgls(b[0], 2)
    for k in range(n_test):
        _, gc = plan.cgls(b[k], max_iters)
        gc = gc.cpu().numpy()
        g0 = float(gc[0])
        with torch.no_grad():
            x0 = net(z[k:k + 1])[0]
        _, gw = plan.cgls(b[k], max_iters, x0=x0)
        gwn = gw.cpu().numpy()
        kc, kw = iterations_to(gc, g0, tol), iterations_to(gwn, g0, tol)
        loose.append([(iterations_to(gc, g0, t), iterations_to(gwn, g0, t)) for t in (1e-2, 1e-3)])
        start.append(float(np.sqrt(gwn[0] / g0)))
        tc = tw = None
        if kc is not None:
            a, e = ev()
            a.record()
            plan.cgls(b[k], kc, history=False)
            e.record()
            e.synchronize()
            tc = a.elapsed_time(e)
        if kw is not None:
            a, e = ev()
            a.record()
            with torch.no_grad():
                x0 = net(z[k:k + 1])[0]
            plan.cgls(b[k], kw, x0=x0, history=False)
            e.record()
            e.synchronize()
            tw = a.elapsed_time(e)
        rows.append((kc, kw, tc, tw))
    res = summarize(rows)
    res["tol"] = tol
    res["warm_start_rel_residual"] = {"median": float(np.median(start)), "q25": float(np.percentile(start, 25)),
                                      "q75": float(np.percentile(start, 75))}
    for j, t in enumerate((1e-2, 1e-3)):
        kc = [r[j][0] for r in loose]
        kw = [r[j][1] for r in loose]
        res[f"iters_at_{t:g}"] = {"cold_median": float(np.median([k for k in kc if k is not None])),
                                  "warm_median": float(np.median([k for k in kw if k is not None]))}
    log(json.dumps(res))
    return res, rows


def summarize(rows):
    def q(v):
        v = np.asarray([x for x in v if x is not None], dtype=np.float64)
        if v.size == 0:
            return None
        return {"median": float(np.median(v)), "q25": float(np.percentile(v, 25)), "q75": float(np.percentile(v, 75))}
    kc, kw, tc, tw = zip(*rows)
    both = [(a, b) for a, b in zip(tc, tw) if a is not None and b is not None]
    return {"samples": len(rows), "reached_cold": sum(x is not None for x in kc),
            "reached_warm": sum(x is not None for x in kw),
            "iters_cold": q(kc), "iters_warm": q(kw), "ms_cold": q(tc), "ms_warm": q(tw),
            "warm_faster_fraction": (sum(b < a for a, b in both) / len(both)) if both else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--out", default="warmstart.pt")
    ap.add_argument("--weights", default=None)
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--n-test", type=int, default=256)
    ap.add_argument("--report", default=None, help="write the evaluation summary (JSON) here")
    ap.add_argument("--cg-steps", type=int, default=0, help="train on the residual after this many CGLS steps")
    ap.add_argument("--init", default=None, help="continue from these weights")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=16)
    a = ap.parse_args()
    if a.cmd == "train":
        init = load_net(a.init) if a.init else None
        net, meta = train(n_train=a.n_train, epochs=a.epochs, cg_steps=a.cg_steps, init=init, lr=a.lr,
                          batch=a.batch)
        save(net, meta, a.out)
        print(json.dumps(meta))
    else:
        net, meta = load_net(a.weights)
        res, _ = evaluate(net, meta, n_test=a.n_test)
        if a.report:
            with open(a.report, "w") as f:
                json.dump({"meta": meta, "eval": res}, f, indent=1)


if __name__ == "__main__":
    main()
