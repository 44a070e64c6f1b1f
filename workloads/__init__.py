"""Seeded synthetic inputs for the spline x-ray projector.

This module is shared by the tests, the smoke check and the benchmark, and by
both sides of every parity check (the CUDA path and the FP64 oracle).  It holds
no arithmetic of the method: it only draws coefficients (ellipse phantoms),
acquisition parameters (view angles, detector offsets, distances, point pairs)
and noise.  Turning those parameters into lines and projections is the job of
each side separately.

Phantom recipe: ellipse e has centre r = R sqrt(U), angle 2 pi U (a point
uniform in the disc of radius R), semi-axes U[lo, hi] each, rotation U[0, pi)
and additive intensity U[-0.5, 1.0], drawn in that order with
``numpy.random.default_rng(seed)``; a coefficient is the sum of the
intensities of the ellipses that contain its grid node.  Sizes scale with
N/64 relative to the 64 x 64 case.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "ellipse_phantom", "Geometry", "Workload", "workload", "crop_workload",
    "random_lines_circle", "poisson_counts", "transmission_data", "batch_instance",
    "warmstart_params", "ellipse_images_torch",
]


def ellipse_phantom(n: int, n_ellipses: int, seed: int, radius: float,
                    axes: tuple[float, float], h: float = 1.0) -> np.ndarray:
    """float32 [n][n] coefficients sampled at the grid nodes.

    Node (i, j) is at ((i - (n-1)/2) h, (j - (n-1)/2) h); rows are j."""
    rng = np.random.default_rng(seed)
    c = (np.arange(n) - 0.5 * (n - 1)) * h
    X, Y = np.meshgrid(c, c, indexing="xy")  # X[j, i] = x1 of node (i, j)
    out = np.zeros((n, n), dtype=np.float64)
    for _ in range(n_ellipses):
        r = radius * math.sqrt(rng.uniform())
        a = 2.0 * math.pi * rng.uniform()
        x0, y0 = r * math.cos(a), r * math.sin(a)
        ax = rng.uniform(axes[0], axes[1])
        ay = rng.uniform(axes[0], axes[1])
        rot = rng.uniform(0.0, math.pi)
        inten = rng.uniform(-0.5, 1.0)
        dx, dy = X - x0, Y - y0
        u = (dx * math.cos(rot) + dy * math.sin(rot)) / ax
        v = (-dx * math.sin(rot) + dy * math.cos(rot)) / ay
        out[u * u + v * v <= 1.0] += inten
    return out.astype(np.float32)


@dataclass
class Geometry:
    """Acquisition parameters (no lines yet).

    kind 'parallel': lines (view_angle[a], det0 + j*ddet).
    kind 'fan': flat detector; source at dso*(cos b, sin b), detector through
    -dod*(cos b, sin b) along (-sin b, cos b), bin j centre at det0 + j*ddet.
    kind 'points': explicit point pairs src[m], dst[m].
    Ray index = view * n_det + bin for the structured kinds."""
    kind: str
    view_angle: np.ndarray | None = None   # float32 [n_view]
    n_det: int = 0
    det0: float = 0.0
    ddet: float = 1.0
    dso: float = 0.0
    dod: float = 0.0
    src: np.ndarray | None = None           # float32 [m][2]
    dst: np.ndarray | None = None           # float32 [m][2]

    @property
    def n_view(self) -> int:
        return 0 if self.view_angle is None else int(self.view_angle.size)

    @property
    def m(self) -> int:
        if self.kind == "points":
            return int(self.src.shape[0])
        return self.n_view * self.n_det


@dataclass
class Workload:
    name: str
    n: int                 # grid is n x n
    degree: int
    h: float
    geometry: Geometry
    coef: np.ndarray       # float32 [n][n]
    seed: int
    notes: dict = field(default_factory=dict)


def _angles(count: int, span: float) -> np.ndarray:
    return (np.arange(count, dtype=np.float64) * (span / count)).astype(np.float32)


def workload(name: str) -> Workload:
    """The fixed workloads.

    parallel64_linear   64 x 64, degree 1, 90 angles in [0, pi), 96 offsets -48 + b.
    fan512_cubic        512 x 512, degree 3, fan: 720 views in [0, 2 pi),
                        768 bins of width 1 centred on the axis, dso 1000, dod 500.
    parallel256_cubic   256 x 256, degree 3, 360 angles in [0, pi), 384 offsets -192 + j.
    fan256_cubic        fan512_cubic at half size (256 x 256, 360 views x 384 bins,
                        dso 500, dod 250), a small case of the same kernels.
    """
    if name == "parallel64_linear":
        n = 64
        geo = Geometry("parallel", view_angle=_angles(90, math.pi), n_det=96, det0=-48.0, ddet=1.0)
        coef = ellipse_phantom(n, 10, 0, radius=24.0, axes=(2.0, 16.0))
        return Workload(name, n, 1, 1.0, geo, coef, 0)
    if name == "fan512_cubic":
        n = 512
        s = n / 64.0
        geo = Geometry("fan", view_angle=_angles(720, 2.0 * math.pi), n_det=768,
                       det0=-383.5, ddet=1.0, dso=1000.0, dod=500.0)
        coef = ellipse_phantom(n, 30, 1, radius=24.0 * s, axes=(2.0 * s, 16.0 * s))
        return Workload(name, n, 3, 1.0, geo, coef, 1)
    if name == "fan256_cubic":
        n = 256
        s = n / 64.0
        geo = Geometry("fan", view_angle=_angles(360, 2.0 * math.pi), n_det=384,
                       det0=-191.5, ddet=1.0, dso=500.0, dod=250.0)
        coef = ellipse_phantom(n, 30, 2, radius=24.0 * s, axes=(2.0 * s, 16.0 * s))
        return Workload(name, n, 3, 1.0, geo, coef, 2)
    if name == "parallel256_cubic":
        n = 256
        s = n / 64.0
        geo = Geometry("parallel", view_angle=_angles(360, math.pi), n_det=384, det0=-192.0, ddet=1.0)
        coef = ellipse_phantom(n, 20, 4, radius=24.0 * s, axes=(2.0 * s, 16.0 * s))
        return Workload(name, n, 3, 1.0, geo, coef, 4)
    raise KeyError(name)


def crop_workload(base: Workload, n: int, degree: int | None = None, seed: int | None = None) -> Workload:
    """A smaller instance with the same kind of geometry, distances and bin
    counts scaled by n / base.n (used for small parity and gradient checks)."""
    g = base.geometry
    s = n / base.n
    deg = base.degree if degree is None else degree
    sd = base.seed if seed is None else seed
    if g.kind == "fan":
        n_det = max(8, int(round(g.n_det * s)))
        ddet = g.ddet
        geo = Geometry("fan", view_angle=_angles(max(8, int(round(g.n_view * s))), 2.0 * math.pi),
                       n_det=n_det, det0=-0.5 * (n_det - 1) * ddet, ddet=ddet,
                       dso=g.dso * s, dod=g.dod * s)
    elif g.kind == "parallel":
        n_det = max(8, int(round(g.n_det * s)))
        geo = Geometry("parallel", view_angle=_angles(max(8, int(round(g.n_view * s))), math.pi),
                       n_det=n_det, det0=-0.5 * n_det * g.ddet, ddet=g.ddet)
    else:
        raise ValueError(g.kind)
    sc = n / 64.0
    coef = ellipse_phantom(n, 10, sd, radius=24.0 * sc, axes=(2.0 * sc, 16.0 * sc))
    return Workload(f"{base.name}_crop{n}", n, deg, base.h, geo, coef, sd)


def random_lines_circle(m: int, radius: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """m chords with both endpoints at angles U[0, 2 pi) on a circle (float32 [m][2] each)."""
    rng = np.random.default_rng(seed)
    a0 = rng.uniform(0.0, 2.0 * math.pi, m)
    a1 = rng.uniform(0.0, 2.0 * math.pi, m)
    src = np.stack([radius * np.cos(a0), radius * np.sin(a0)], axis=1).astype(np.float32)
    dst = np.stack([radius * np.cos(a1), radius * np.sin(a1)], axis=1).astype(np.float32)
    return src, dst


def poisson_counts(expected: np.ndarray, seed: int) -> np.ndarray:
    """Poisson draws with the given means (float64 in, float64 out)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.asarray(expected, dtype=np.float64)).astype(np.float64)


def transmission_data(expected: np.ndarray, seed: int, peak: float = 3.0, I0: float = 1e4):
    """Noisy line integrals for a transmission scan of a noiseless sinogram.

    Scale kappa = peak / max(expected) (so the largest attenuation is
    ``peak``); counts ~ Poisson(I0 exp(-kappa expected)); returned data
    -ln(max(counts, 1) / I0) / kappa (float64), in the units of ``expected``,
    and kappa."""
    e = np.asarray(expected, dtype=np.float64)
    top = float(e.max())
    kappa = peak / top if top > 0 else 1.0
    counts = poisson_counts(I0 * np.exp(-kappa * e), seed)
    return -np.log(np.maximum(counts, 1.0) / I0) / kappa, kappa


def batch_instance(i: int, scale: float = 1.0) -> Workload:
    """Instance i of the uneven batch (seed 1000 + i).

    N = round(exp U[ln 128, ln 1024] * scale), degree U{0..3}; one instance in
    eight is a free line list of M ~ U[1e5, 1e6] * scale^2 chords with both
    endpoints at angles U[0, 2 pi) on the circle of radius 0.75 N; the others
    are parallel or fan beams (probability 1/2 each) with U{180..1440} * scale
    views and round(1.5 N) bins of width 1 (fan: dso = 1000 N/512,
    dod = 500 N/512).  The phantom has 10 ellipses scaled to the grid."""
    rng = np.random.default_rng(1000 + i)
    n = max(16, int(round(math.exp(rng.uniform(math.log(128), math.log(1024))) * scale)))
    degree = int(rng.integers(0, 4))
    s = n / 64.0
    coef = ellipse_phantom(n, 10, 1000 + i, radius=24.0 * s, axes=(2.0 * s, 16.0 * s))
    if i % 8 == 7:
        m = max(1000, int(rng.uniform(1e5, 1e6) * scale * scale))
        src, dst = random_lines_circle(m, 0.75 * n, 1000 + i)
        geo = Geometry("points", src=src, dst=dst)
    else:
        n_view = max(8, int(round(rng.integers(180, 1441) * scale)))
        n_det = int(round(1.5 * n))
        if rng.uniform() < 0.5:
            geo = Geometry("parallel", view_angle=_angles(n_view, math.pi), n_det=n_det,
                           det0=-0.5 * (n_det - 1), ddet=1.0)
        else:
            geo = Geometry("fan", view_angle=_angles(n_view, 2.0 * math.pi), n_det=n_det,
                           det0=-0.5 * (n_det - 1), ddet=1.0, dso=1000.0 * n / 512.0, dod=500.0 * n / 512.0)
    return Workload(f"batch{i}", n, degree, 1.0, geo, coef, 1000 + i)


def warmstart_params(seed: int, n: int = 256):
    """Phantom and dose of one sample of the warm-start data set.

    numpy default_rng(seed): number of ellipses U{5..40}, then per ellipse
    the recipe of :func:`ellipse_phantom` (centre, semi-axes, rotation,
    intensity) at the scale n/64, then the dose I0 log-uniform in
    [1e3, 1e5].  Returns (params float64 [k][6] = x0, y0, ax, ay, rot,
    intensity; I0).  Training seeds are 1e6 + i, held-out seeds 2e6 + i."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(5, 41))
    s = n / 64.0
    radius, lo, hi = 24.0 * s, 2.0 * s, 16.0 * s
    out = np.empty((k, 6))
    for e in range(k):
        r = radius * math.sqrt(rng.uniform())
        a = 2.0 * math.pi * rng.uniform()
        out[e, 0], out[e, 1] = r * math.cos(a), r * math.sin(a)
        out[e, 2] = rng.uniform(lo, hi)
        out[e, 3] = rng.uniform(lo, hi)
        out[e, 4] = rng.uniform(0.0, math.pi)
        out[e, 5] = rng.uniform(-0.5, 1.0)
    I0 = float(math.exp(rng.uniform(math.log(1e3), math.log(1e5))))
    return out, I0


def ellipse_images_torch(params_list, n: int, device, h: float = 1.0):
    """Rasterise ellipse parameter sets (see :func:`warmstart_params`) at the
    nodes of an n x n grid, as :func:`ellipse_phantom` does, on `device`:
    float32 [len(params_list)][n][n]."""
    import torch
    c = (torch.arange(n, device=device, dtype=torch.float64) - 0.5 * (n - 1)) * h
    Y, X = torch.meshgrid(c, c, indexing="ij")
    out = torch.zeros((len(params_list), n, n), device=device, dtype=torch.float64)
    for b, prm in enumerate(params_list):
        P = torch.as_tensor(prm, device=device, dtype=torch.float64)
        x0, y0, ax, ay, rot, inten = (P[:, k, None, None] for k in range(6))
        dx, dy = X - x0, Y - y0
        u = (dx * torch.cos(rot) + dy * torch.sin(rot)) / ax
        v = (-dx * torch.sin(rot) + dy * torch.cos(rot)) / ay
        out[b] = (inten * (u * u + v * v <= 1.0)).sum(dim=0)
    return out.float()
