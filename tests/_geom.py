"""Helpers that hand the same seeded acquisition parameters to both sides:
the CUDA library (device tensors through the C ABI) and the FP64 oracle
(which expands the geometry itself)."""
from __future__ import annotations

import numpy as np

import oracle
import workloads


def oracle_lines(geo: workloads.Geometry):
    if geo.kind == "parallel":
        return oracle.lines_parallel(geo.view_angle.astype(np.float64), geo.n_det, geo.det0, geo.ddet)
    if geo.kind == "fan":
        return oracle.lines_fan(geo.view_angle.astype(np.float64), geo.dso, geo.dod, geo.n_det,
                                geo.det0, geo.ddet)
    if geo.kind == "points":
        return oracle.lines_points(geo.src.astype(np.float64), geo.dst.astype(np.float64))
    raise ValueError(geo.kind)


def device_lines(geo: workloads.Geometry, device):
    import torch
    import paper_2503_20907_gb300 as sp
    if geo.kind == "parallel":
        return sp.Lines.parallel(torch.from_numpy(geo.view_angle).to(device), geo.n_det, geo.det0, geo.ddet)
    if geo.kind == "fan":
        return sp.Lines.fan(torch.from_numpy(geo.view_angle).to(device), geo.dso, geo.dod, geo.n_det,
                            geo.det0, geo.ddet)
    if geo.kind == "points":
        return sp.Lines.points(torch.from_numpy(geo.src).to(device), torch.from_numpy(geo.dst).to(device))
    raise ValueError(geo.kind)


def rel_l2(got, ref) -> float:
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))
