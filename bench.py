#!/usr/bin/env python
"""Throughput of the spline x-ray projector on one GB300.

Workload: 512 x 512 cubic B-spline grid, fan beam with 720 views x 768 bins
(dso 1000, dod 500), 30-ellipse seeded phantom.  One step is one pass of the
whole hot path over that batch: line setup, footprint tables, forward
projection and adjoint, each a call of the C ABI (spline_plan_prepare,
spline_plan_fwd, spline_plan_adj).  value = lines x steps / time, in Mrays/s
(one ray counted once per forward+adjoint pair).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (launched by torch.distributed.run) every rank runs its own
instance (independent replicas, weak scaling); value is the sum over ranks
divided by the slowest rank's time.  --impl reference times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s fwd+adj at 512² cubic fan-beam (% roofline); learned-vs-cold CG time to 1e-4"
UNIT = "Mrays/s"
WORKLOAD = "fan512_cubic"
FP32_LANES_PER_SM = 128
KERNELS_PER_STEP = 6   # line setup with tables (one fused kernel), transpose + forward strip, adjoint strip (fixed-point chunks, then float chunks) + transposed add
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu
# capture of these kernel versions on this workload); set to None whenever the
# kernels change until they are captured again.
TRAFFIC = {"fan512_cubic": {"spline_fwd": 770800896, "spline_adj": 772362240}}   # re-captured after each kernel change
CG_ITERS = 100
CG_MAX_ITERS = 400   # cap of the run to the tolerance
CG_TOL = 1e-4
FLOPS_PER_PAIR = lambda n: 2 * (2 * n + 3)   # noqa: E731  (2n+1 Horner FMAs, 1 offset, 1 accumulate)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cg", action="store_true", help="skip the CGLS timing (not part of the step)")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven-batch timing (not part of the step)")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start timing (not part of the step)")
    ap.add_argument("--no-schemes", action="store_true", help="skip timing the adjoint schemes (not part of the step)")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="size scale of the uneven batch")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="fan512_cubic (the benchmark) or fan256_cubic (small profiling case)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """SM clock and clock-event reasons while the timed region runs: NVML
    queries (read-only, through ctypes) every 5 ms from a thread, else
    nvidia-smi every 50 ms.  Only samples taken between start() and stop()
    count."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8 | 0x80, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None
        self.lib, self.handle, self.thread, self.rows, self.max_mhz = None, None, None, [], None
        self._stop = False
        self._open_nvml()

    def _open_nvml(self):
        import ctypes
        lib = None
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if lib is None or lib.nvmlInit_v2() != 0:
            return
        h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.index)
            bus = f"{pr.pci_domain_id:x}:{pr.pci_bus_id:x}:{pr.pci_device_id:x}.0".encode()
            ok = lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) == 0
        except Exception:
            ok = False
        if not ok:
            ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) == 0
        if not ok:
            return
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) != 0:
            return
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
        if self.reasons_fn is None:
            return
        self.lib, self.handle, self.max_mhz = lib, h, float(mx.value)

    def _sample_loop(self):
        import ctypes
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop:
            if (self.lib.nvmlDeviceGetClockInfo(self.handle, ctypes.c_int(1), ctypes.byref(clk)) == 0 and
                    self.reasons_fn(self.handle, ctypes.byref(rs)) == 0):
                self.rows.append((float(clk.value), int(rs.value)))
            time.sleep(0.005)

    def start(self):
        if self.lib is not None:
            import threading
            self._stop = False
            self.thread = threading.Thread(target=self._sample_loop, daemon=True)
            self.thread.start()
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self._stop = True
            self.thread.join(timeout=5)
            if not self.rows:
                return None
            reasons = sorted({k for _, r in self.rows for k, bit in self.BITS.items() if r & bit})
            return {"sm_mhz": statistics.median(c for c, _ in self.rows), "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(self.rows), "source": "nvml, 5 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi, 50 ms"}


# ------------------------------------------------------------------ distributed
def dist_setup(n_gpus):
    """One process per GPU under torch.distributed.run (NCCL); without a GPU
    (the reference arm, or host-side tests) the ranks use gloo."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
        return dist.get_rank(), ws, local
    return 0, 1, 0


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle
def cpu_model() -> str:
    """The host CPU's model name: lscpu's, else /proc/cpuinfo's "model name",
    else its implementer and part codes (Arm), else the platform string."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                name = line.split(":", 1)[1].strip()
                if name and name != "-":
                    return name
    except Exception:
        pass
    try:
        impl = part = None
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            k, v = k.strip().lower(), v.strip()
            if k == "model name" and v:
                return v
            if k == "cpu implementer":
                impl = v
            if k == "cpu part":
                part = v
        if impl or part:
            return f"arm implementer {impl} part {part}"
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_sample(wl, nf: int = 6000, npix: int = 160, threads: int = 0):
    """Time the FP64 oracle, as it stands, on a bounded sample of the
    workload and scale to the full job: forward on nf random lines, adjoint
    on npix random nodes (pixel-driven over every line); threads = 0: all
    host cores."""
    import numpy as np
    import oracle
    geo = wl.geometry
    th, yy = oracle.lines_fan(geo.view_angle.astype(np.float64), geo.dso, geo.dod, geo.n_det,
                              geo.det0, geo.ddet)
    g = oracle.Grid(wl.n, wl.n, wl.degree, wl.h)
    rng = np.random.default_rng(7)
    ridx = np.sort(rng.choice(th.size, nf, replace=False))
    t0 = time.perf_counter()
    oracle.forward(g, wl.coef, th[ridx], yy[ridx], threads=threads)
    tf = time.perf_counter() - t0
    p = rng.uniform(-1, 1, th.size)
    pix = np.sort(rng.choice(wl.n * wl.n, npix, replace=False))
    t0 = time.perf_counter()
    oracle.adjoint_pixels(g, p, th, yy, pix, threads=threads)
    ta = time.perf_counter() - t0
    m = th.size
    t_full = tf * m / nf + ta * (wl.n * wl.n) / npix
    return {"value": m / t_full / 1e6, "unit": UNIT, "cores": threads or oracle.max_threads(), "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"forward on {nf} of {m} lines ({tf:.2f} s), adjoint on {npix} of {wl.n * wl.n} nodes "
                      f"({ta:.2f} s), scaled to the full job ({t_full:.0f} s)",
            "seconds": tf + ta}


def oracle_small_full(threads: int):
    """The FP64 oracle's whole forward and adjoint on the 64 x 64 linear
    parallel workload (8,640 lines), timed on `threads` host cores."""
    import numpy as np
    import oracle
    import workloads
    wl = workloads.workload("parallel64_linear")
    geo = wl.geometry
    th, yy = oracle.lines_parallel(geo.view_angle.astype(np.float64), geo.n_det, geo.det0, geo.ddet)
    g = oracle.Grid(wl.n, wl.n, wl.degree, wl.h)
    t0 = time.perf_counter()
    s = oracle.forward(g, wl.coef, th, yy, threads=threads)
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.adjoint(g, s, th, yy, threads=threads)
    ta = time.perf_counter() - t0
    return {"workload": "parallel64_linear (64x64 linear, 90 x 96 lines), whole forward and adjoint",
            "cores": threads, "fwd_s": tf, "adj_s": ta, "mrays_per_s": th.size / (tf + ta) / 1e6}


def cg_oracle_sample(sp, dev, n=64, iters=100):
    """CPU baseline of the reconstruction step, and the GPU iterates against
    it: FP64 oracle CGLS (100 iterations) on the 64 x 64 crop of the 512^2
    cubic fan scan (transmission data, Poisson seed 3), timed on the host
    cores; then the relative L2 error of each GPU iterate x_k (spline_plan_cgls
    run k iterations from x_0 = 0) against the oracle's x_k, k = 1..100, in
    the image and in the data (||A (x_k - x_k^orc)|| / ||A x_k^orc||, A the
    oracle's forward), and both relative normal-equation residuals."""
    import numpy as np
    import torch
    import oracle
    from oracle.cgls import cgls
    import workloads
    W = workloads.crop_workload(workloads.workload(WORKLOAD), n)
    geo = W.geometry
    th, yy = oracle.lines_fan(geo.view_angle.astype(np.float64), geo.dso, geo.dod, geo.n_det, geo.det0, geo.ddet)
    og = oracle.Grid(W.n, W.n, W.degree, W.h)
    b, _ = workloads.transmission_data(oracle.forward(og, W.coef.astype(np.float64), th, yy), seed=3)
    b32 = b.astype(np.float32)
    nt = os.cpu_count() or 1   # explicit: an earlier one-core sample leaves OpenMP at one thread
    t0 = time.perf_counter()
    _, gam_o, kept = cgls(lambda x: oracle.forward(og, x, th, yy, threads=nt),
                          lambda p: oracle.adjoint(og, p, th, yy, threads=nt),
                          b32.astype(np.float64), np.zeros((W.n, W.n)), iters, keep=range(1, iters + 1))
    t_orc = time.perf_counter() - t0
    plan = sp.Plan(sp.Grid(W.n, W.n, W.degree, W.h),
                   sp.Lines.fan(torch.from_numpy(geo.view_angle).to(dev), geo.dso, geo.dod, geo.n_det,
                                geo.det0, geo.ddet))
    bt = torch.from_numpy(b32).to(dev)
    err, err_data = [], []
    for k in range(1, iters + 1):
        x, _ = plan.cgls(bt, k, history=False)
        ref = kept[k]
        d = x.cpu().numpy().astype(np.float64) - ref
        err.append(float(np.linalg.norm(d) / np.linalg.norm(ref)))
        err_data.append(float(np.linalg.norm(oracle.forward(og, d, th, yy, threads=nt))
                              / np.linalg.norm(oracle.forward(og, ref, th, yy, threads=nt))))
    _, gam_g = plan.cgls(bt, iters)
    gam_g = gam_g.cpu().numpy()
    plan.close()
    at = [k for k in (1, 2, 5, 10, 20, 50, 100) if k <= iters]
    return {"workload": f"64x64 crop of {WORKLOAD} ({th.size} lines), transmission data, Poisson seed 3, x0 = 0",
            "oracle_seconds_100_iters": t_orc, "cores": nt,
            "rel_err_vs_oracle_per_iter": [float(f"{e:.3g}") for e in err],
            "rel_data_err_vs_oracle_per_iter": [float(f"{e:.3g}") for e in err_data],
            "max_rel_err_k_le_5": max(err[:5]),
            "rel_residual_normal_eq": {str(k): {"gpu": float(f"{np.sqrt(gam_g[k] / gam_g[0]):.4g}"),
                                                "oracle": float(f"{np.sqrt(gam_o[k] / gam_o[0]):.4g}")}
                                       for k in at}}


def run_reference(args, rank, ws):
    if rank != 0:
        return
    import workloads
    wl = workloads.workload(WORKLOAD)
    times = []
    for k in range(args.warmup + args.steps):
        cb = oracle_sample(wl)
        if k >= args.warmup:
            times.append(cb)
    value = statistics.mean(c["value"] for c in times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(c["seconds"] for c in times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "grid": wl.n, "degree": wl.degree,
                                            "geometry": "fan 720 views x 768 bins, dso 1000, dod 500",
                                            "sample": "bounded sample per step, scaled to the full job"},
            "cpu_baseline": {k: times[-1][k] for k in ("value", "unit", "cores", "kind", "sample", "cpu_model")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU
def run_batch(args, sp, dev, stream, count=64):
    """The uneven batch (64 seeded instances, one CUDA graph per direction),
    autotuned; lines per second over forward + adjoint of all instances."""
    import torch
    import workloads

    ws_ = [workloads.batch_instance(i, args.batch_scale) for i in range(count)]
    grids, lines, coefs = [], [], []
    for w in ws_:
        geo = w.geometry
        grids.append(sp.Grid(w.n, w.n, w.degree, w.h))
        if geo.kind == "points":
            lines.append(sp.Lines.points(torch.from_numpy(geo.src).to(dev), torch.from_numpy(geo.dst).to(dev)))
        elif geo.kind == "parallel":
            lines.append(sp.Lines.parallel(torch.from_numpy(geo.view_angle).to(dev), geo.n_det, geo.det0, geo.ddet))
        else:
            lines.append(sp.Lines.fan(torch.from_numpy(geo.view_angle).to(dev), geo.dso, geo.dod, geo.n_det,
                                      geo.det0, geo.ddet))
        coefs.append(torch.from_numpy(w.coef).to(dev))
    batch = sp.Batch(grids, lines)
    sinos = batch.fwd(coefs)
    backs = batch.adj(sinos)
    paths = batch.autotune(coefs, sinos)
    for _ in range(3):
        batch.fwd(coefs, sinos)
        batch.adj(sinos, backs)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    a.record(stream)
    for _ in range(reps):
        batch.fwd(coefs, sinos)
        batch.adj(sinos, backs)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    m_tot = sum(L.m for L in lines)
    out = {"workload": f"{count} seeded uneven instances (sizes 128..1024 x {args.batch_scale:g}, degrees 0..3, "
                       "parallel/fan views, 1 in 8 a free line list)",
           "lines": m_tot, "ms_fwd_adj": ms, "mrays_per_s": m_tot / (ms / 1000.0) / 1e6,
           "strip_fwd": sum(1 for f, _ in paths if f == 1), "strip_adj": sum(1 for _, x in paths if x == 1),
           "graphs": "one CUDA graph per direction, replayed"}
    batch.close()
    return out


def run_warmstart(sp, dev, n_test=256, tol=1e-4):
    """Learned-vs-cold CGLS to a relative normal-equation residual of 1e-4 on
    held-out samples (256^2 cubic, parallel 360 x 384, Poisson data), with the
    committed network; times include the network's forward."""
    from paper_2503_20907_gb300 import warmstart as wsm
    net, meta = wsm.load_net(wsm.DEFAULT_WEIGHTS, dev)
    res, _ = wsm.evaluate(net, meta, n_test=n_test, tol=tol, log=lambda *_: None)
    import torch
    zz = torch.zeros(1, 256, 256, device=dev)
    with torch.no_grad():
        for _ in range(3):
            net(zz)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            net(zz)
        b.record()
        b.synchronize()
    res["network_ms"] = a.elapsed_time(b) / 10
    res["workload"] = ("256x256 cubic, parallel 360 x 384, held-out phantoms (seeds 2e6+i), Poisson data at "
                       "log-uniform dose; committed weights")
    return res


def run_ours(args, rank, ws, local):
    import numpy as np
    import torch

    import paper_2503_20907_gb300 as sp
    import workloads

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    props = torch.cuda.get_device_properties(dev)
    wl = workloads.workload(args.workload)
    geo = wl.geometry
    grid = sp.Grid(wl.n, wl.n, wl.degree, wl.h)
    view = torch.from_numpy(geo.view_angle).to(dev)
    lines = sp.Lines.fan(view, geo.dso, geo.dod, geo.n_det, geo.det0, geo.ddet)
    M = lines.m
    coef = torch.from_numpy(wl.coef).to(dev)
    sino = torch.empty(M, device=dev)
    back = torch.empty(wl.n, wl.n, device=dev)
    plan = sp.Plan(grid, lines, prepare=True)
    pairs = int(sp.spline_visited(grid, lines).to(torch.int64).sum().item())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()
    # FP32 throughput of this GPU, measured with the library's FMA-chain
    # probe (scalar and packed FMAs; the roofline takes the larger), before
    # the timed region
    peak_ffma, _ = sp.fp32_peak(False, stream)
    peak_ffma2, _ = sp.fp32_peak(True, stream)

    def step(ev=None):
        if ev: ev[0].record(stream)
        plan.prepare(stream)
        if ev: ev[1].record(stream)
        plan.fwd(coef, sino, stream)
        if ev: ev[2].record(stream)
        plan.adj(sino, back, stream)
        if ev: ev[3].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    barrier(ws)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))          # L2 flush between timed steps (outside the events)
        step(evs[k])
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    prep = [e[0].elapsed_time(e[1]) for e in evs]
    fwd = [e[1].elapsed_time(e[2]) for e in evs]
    adj = [e[2].elapsed_time(e[3]) for e in evs]
    tot = sum(e[0].elapsed_time(e[3]) for e in evs) / 1000.0
    tmax = allreduce_max(tot, ws)
    slow_rows = plan.slow_rows()

    # end to end through the public API with host buffers
    coef_h = torch.from_numpy(wl.coef).pin_memory()
    view_h = torch.from_numpy(geo.view_angle).pin_memory()
    sino_h = torch.empty(M, dtype=torch.float32).pin_memory()
    back_h = torch.empty(wl.n, wl.n, dtype=torch.float32).pin_memory()
    coef_d = torch.empty_like(coef)

    def e2e_step():
        coef_d.copy_(coef_h, non_blocking=True)
        view.copy_(view_h, non_blocking=True)
        plan.prepare(stream)
        plan.fwd(coef_d, sino, stream)
        plan.adj(sino, back, stream)
        sino_h.copy_(sino, non_blocking=True)
        back_h.copy_(back, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
    e2e_t = allreduce_max(sum(e_ms) / 1000.0, ws)
    h2d = coef_h.numel() * 4 + view_h.numel() * 4
    d2h = sino_h.numel() * 4 + back_h.numel() * 4

    # Adjoint schemes timed on this workload and on the 256^2 cubic parallel
    # beam (per-view tables): strip scatter, warp-per-line scatter, pixel-driven
    # gather (spline_plan_autotune's measurements)
    schemes = {}
    if not args.no_schemes:
        for name in (wl.name, "parallel256_cubic"):
            w2 = wl if name == wl.name else workloads.workload(name)
            g2 = w2.geometry
            if g2.kind == "fan":
                l2 = sp.Lines.fan(torch.from_numpy(g2.view_angle).to(dev), g2.dso, g2.dod, g2.n_det, g2.det0, g2.ddet)
            else:
                l2 = sp.Lines.parallel(torch.from_numpy(g2.view_angle).to(dev), g2.n_det, g2.det0, g2.ddet)
            p2 = sp.Plan(sp.Grid(w2.n, w2.n, w2.degree, w2.h), l2, prepare=True)
            c2 = torch.from_numpy(w2.coef).to(dev)
            s2 = p2.fwd(c2)
            _, a_path, ms = p2.autotune(c2, s2)
            schemes[name] = {"adj_strip_scatter_ms": ms[2], "adj_warp_scatter_ms": ms[3], "adj_gather_ms": ms[4],
                             "fwd_strip_ms": ms[0], "fwd_warp_ms": ms[1],
                             "adj_choice": {1: "strip scatter", 2: "warp scatter", 3: "gather"}.get(a_path)}
            p2.close()

    # A free line list: 10^6 random chords (both endpoints uniform on the
    # circle of radius 0.75 N) on the same grid, on the strip kernels through
    # their sorted order against the warp-per-line kernels (autotuner timings),
    # and its prepare (line setup, tables, sort) timed alone.
    free = None
    if not args.no_schemes:
        src, dst = workloads.random_lines_circle(1_000_000, 0.75 * wl.n, 17)
        lf = sp.Lines.points(torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev))
        pf = sp.Plan(grid, lf, prepare=True)
        sf = pf.fwd(coef)
        f_path, a_path, ms = pf.autotune(coef, sf)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pt = []
        for _ in range(5):
            e0.record(stream)
            pf.prepare(stream)
            e1.record(stream)
            e1.synchronize()
            pt.append(e0.elapsed_time(e1))
        pf.set_paths(1, 1)
        pf.fwd(coef)
        pf.adj(sf)
        torch.cuda.synchronize()
        free = {"workload": f"1e6 random chords on the {wl.n}^2 cubic grid (endpoints on the circle of radius 0.75 N)",
                "fwd_strip_ms": ms[0], "fwd_warp_ms": ms[1], "adj_strip_ms": ms[2], "adj_warp_ms": ms[3],
                "prepare_ms": statistics.median(pt[1:]), "slow_rows": pf.slow_rows(),
                "mrays_per_s_fwd_adj": 1.0 / (1e-3 * (min(ms[0], ms[1]) + min(ms[2], ms[3]))),
                "choice": [{1: "strip", 2: "warp"}.get(f_path), {1: "strip", 2: "warp", 3: "gather"}.get(a_path)]}
        pf.close()

    # The same step with row records kept by the plan (written by prepare,
    # read by both projections), as iterative solvers use it.
    rec = None
    plan_r = sp.Plan(grid, lines, prepare=True, records=True)
    if plan_r.record_bytes() > 0:
        def step_r(ev):
            ev[0].record(stream)
            plan_r.prepare(stream)
            ev[1].record(stream)
            plan_r.fwd(coef, sino, stream)
            ev[2].record(stream)
            plan_r.adj(sino, back, stream)
            ev[3].record(stream)
        evr = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        for k in range(3):
            step_r(evr[0])
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            step_r(evr[k])
        torch.cuda.synchronize()
        rp_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evr)
        rf_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evr)
        ra_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in evr)
        rec = {"record_bytes": plan_r.record_bytes(),
               "stage_ms": {"prepare": rp_ms, "fwd": rf_ms, "adj": ra_ms},
               "mrays_per_s_step": M / ((rp_ms + rf_ms + ra_ms) / 1000.0) / 1e6,
               "mrays_per_s_fwd_adj": M / ((rf_ms + ra_ms) / 1000.0) / 1e6}
    else:
        plan_r.close()
        plan_r = None

    # CGLS on transmission data of the same scan (the reconstruction step),
    # on the plan with row records when it has them
    cg = None
    if not args.no_cg:
        cgplan = plan_r if plan_r is not None else plan
        plan.fwd(coef, sino, stream)
        b_np, _ = workloads.transmission_data(sino.cpu().numpy(), seed=3)
        b_cg = torch.from_numpy(b_np.astype(np.float32)).to(dev)
        cgplan.cgls(b_cg, 2)                       # allocates the plan's CG workspace
        torch.cuda.synchronize()

        def timed_cgls(iters, history=True):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, gam = cgplan.cgls(b_cg, iters, history=history)
            b.record(stream)
            b.synchronize()
            return a.elapsed_time(b), gam

        ms100, gam = timed_cgls(CG_ITERS)
        g = gam.cpu().numpy()
        # the same solve run on until the relative normal-equation residual
        # reaches the tolerance, then timed for exactly that many iterations
        _, gam_long = timed_cgls(CG_MAX_ITERS)
        gl = gam_long.cpu().numpy()
        k_tol = next((k for k in range(len(gl)) if np.sqrt(gl[k] / gl[0]) < CG_TOL), None)
        ms_tol = timed_cgls(k_tol, history=False)[0] if k_tol else None
        cg = {"workload": f"{wl.name} transmission data (peak attenuation 3, I0 1e4, Poisson seed 3), x0 = 0",
              "iters": CG_ITERS, "ms_per_iter": ms100 / CG_ITERS,
              "rel_residual_normal_eq": float(np.sqrt(g[-1] / g[0])),
              "tol": CG_TOL, "iters_to_tol": k_tol, "ms_to_tol": ms_tol,
              "rel_residual_at": {str(k): float(np.sqrt(gl[k] / gl[0])) for k in (10, 50, 100, 150, 200, 300)
                                  if k < len(gl)},
              "kernels_per_iter": 8, "row_records": cgplan.record_bytes() > 0}

    batch = None if args.no_batch else run_batch(args, sp, dev, stream)
    warm = None if args.no_warm else run_warmstart(sp, dev)

    if rank != 0:
        return
    value = ws * M * args.steps / tmax / 1e6
    fwd_ms, adj_ms, prep_ms = statistics.mean(fwd), statistics.mean(adj), statistics.mean(prep)
    dom_name, dom_ms = ("spline_fwd", fwd_ms) if fwd_ms >= adj_ms else ("spline_adj", adj_ms)
    flops = FLOPS_PER_PAIR(wl.degree) * pairs
    achieved = flops / (dom_ms / 1000.0) / 1e12
    max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak_derived = props.multi_processor_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    peak = max(peak_ffma, peak_ffma2)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "grid": wl.n, "degree": wl.degree,
                   "geometry": f"fan {geo.n_view} views x {geo.n_det} bins, dso {geo.dso:g}, dod {geo.dod:g}",
                   "lines": M,
                   "phantom": "30 seeded ellipses", "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{ws}"},
        "stage_ms": {"prepare": prep_ms, "fwd": fwd_ms, "adj": adj_ms},
        "per_direction": {d: {"mrays_per_s": M / t / 1e3, "basis_evals_per_s": pairs / (t / 1000.0)}
                          for d, t in (("fwd", fwd_ms), ("adj", adj_ms))},
        "pairs_per_direction": pairs,
        "slow_rows": slow_rows,
        "basis_evals_per_s": 2 * pairs * args.steps / (tot) if tot > 0 else None,
        "roofline": {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (TRAFFIC.get(wl.name) or {}).get(dom_name),
                     "peak_source": "measured: independent FMA chains on every SM (sp_fp32_peak), "
                                    "the larger of scalar and packed",
                     "peak_measured": {"ffma": peak_ffma, "ffma2": peak_ffma2},
                     "peak_derived": {"value": peak_derived,
                                      "source": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 "
                                                f"lanes x 2 x {max_mhz:.0f} MHz max SM clock"},
                     "flops_per_pair": FLOPS_PER_PAIR(wl.degree)},
        "e2e": {"value": M * args.steps / e2e_t / 1e6 * ws, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clocks,
        "wall_s": wall,
    }
    if schemes:
        line["adjoint_schemes"] = schemes
    if free is not None:
        line["free_line_list"] = free
    if rec is not None:
        line["with_row_records"] = rec
    if cg is not None:
        line["cg"] = cg
    if batch is not None:
        line["batch"] = batch
    if warm is not None:
        line["warm_start"] = warm
    if ws == 1 and not args.no_cpu_baseline and wl.name == WORKLOAD:
        ncpu = os.cpu_count() or 1
        cb = oracle_sample(wl, nf=120000, npix=1600, threads=ncpu)   # ~10 s on 16 host cores
        cb.pop("seconds", None)
        if cg is not None:
            line["cg"]["vs_oracle_cgls"] = cg_oracle_sample(sp, dev)
        one = oracle_sample(wl, nf=4000, npix=60, threads=1)   # ~5 s on one core
        cb["one_core"] = {"value": one["value"], "sample": one["sample"]}
        cb["small_full"] = [oracle_small_full(ncpu), oracle_small_full(1)]
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, ws, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_ours(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
