"""The seeded input generators that both sides of every parity check use:
the recipe they state (sizes of the named workloads, the ellipse phantom's
geometry, the uneven batch's ranges, chords on a circle, transmission data)
and their determinism.  Host only, no projector arithmetic."""
import math

import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("name,n,degree,kind,m", [
    ("parallel64_linear", 64, 1, "parallel", 90 * 96),
    ("fan512_cubic", 512, 3, "fan", 720 * 768),
    ("fan256_cubic", 256, 3, "fan", 360 * 384),
    ("parallel256_cubic", 256, 3, "parallel", 360 * 384),
])
def test_named_workloads(name, n, degree, kind, m):
    w = workloads.workload(name)
    g = w.geometry
    assert (w.n, w.degree, g.kind, g.m) == (n, degree, kind, m)
    assert w.coef.shape == (n, n) and w.coef.dtype == np.float32
    assert np.count_nonzero(w.coef) > 0
    span = math.pi if kind == "parallel" else 2.0 * math.pi
    # float32 angles a span / n_view, a = 0..n_view-1 (rounded once)
    exact = np.arange(g.n_view) * (span / g.n_view)
    assert g.view_angle.dtype == np.float32
    assert np.max(np.abs(g.view_angle.astype(np.float64) - exact)) <= 4e-7
    if kind == "fan":
        # bins of width 1 centred on the axis through the source
        assert g.det0 == -0.5 * (g.n_det - 1) and g.ddet == 1.0
        assert g.dso / g.dod == 2.0


def test_parallel64_offsets_are_minus_48_plus_b():
    g = workloads.workload("parallel64_linear").geometry
    assert g.det0 == -48.0 and g.ddet == 1.0 and g.n_det == 96


def test_generators_are_deterministic():
    a = workloads.workload("parallel256_cubic").coef
    b = workloads.workload("parallel256_cubic").coef
    assert np.array_equal(a, b)
    assert np.array_equal(workloads.ellipse_phantom(48, 7, 11, 18.0, (2.0, 9.0)),
                          workloads.ellipse_phantom(48, 7, 11, 18.0, (2.0, 9.0)))
    assert not np.array_equal(workloads.ellipse_phantom(48, 7, 11, 18.0, (2.0, 9.0)),
                              workloads.ellipse_phantom(48, 7, 12, 18.0, (2.0, 9.0)))
    s1, d1 = workloads.random_lines_circle(100, 5.0, 3)
    s2, d2 = workloads.random_lines_circle(100, 5.0, 3)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)


def test_ellipse_phantom_geometry():
    # radius 0 puts the centre at the origin and equal axis bounds make a
    # disc: exactly the nodes within that radius carry the one intensity
    n, r = 33, 7.5
    c = workloads.ellipse_phantom(n, 1, 5, radius=0.0, axes=(r, r))
    rng = np.random.default_rng(5)
    rng.uniform(); rng.uniform(); rng.uniform(); rng.uniform(); rng.uniform()   # centre, axes, rotation
    inten = rng.uniform(-0.5, 1.0)
    x = np.arange(n) - 0.5 * (n - 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    inside = X * X + Y * Y <= r * r
    assert np.allclose(c[inside], inten) and np.all(c[~inside] == 0.0)


def test_torch_rasteriser_matches_phantom():
    # the same ellipses drawn in ellipse_phantom's order, rasterised by the
    # batched torch path (warm-start training data): identical images, so
    # node placement (column i = x1, row j = x2) and orientation agree
    torch = pytest.importorskip("torch")
    n, k, seed, h = 40, 6, 21, 0.75
    radius, lo, hi = 12.0, 1.5, 9.0
    rng = np.random.default_rng(seed)
    prm = np.empty((k, 6))
    for e in range(k):
        r = radius * math.sqrt(rng.uniform())
        a = 2.0 * math.pi * rng.uniform()
        prm[e] = (r * math.cos(a), r * math.sin(a), rng.uniform(lo, hi), rng.uniform(lo, hi),
                  rng.uniform(0.0, math.pi), rng.uniform(-0.5, 1.0))
    ref = workloads.ellipse_phantom(n, k, seed, radius=radius, axes=(lo, hi), h=h)
    got = workloads.ellipse_images_torch([prm], n, "cpu", h=h)[0].numpy()
    assert np.array_equal(got, ref)


def test_ellipse_intensities_are_sums_in_range():
    c = workloads.ellipse_phantom(64, 1, 0, radius=24.0, axes=(2.0, 16.0))
    vals = np.unique(c)
    assert len(vals) <= 2 and 0.0 in vals
    assert np.all((vals >= -0.5) & (vals < 1.0))


def test_random_chords_end_on_the_circle():
    src, dst = workloads.random_lines_circle(1000, 12.0, 7)
    assert src.shape == dst.shape == (1000, 2) and src.dtype == np.float32
    assert np.allclose(np.hypot(src[:, 0], src[:, 1]), 12.0, rtol=1e-6)
    assert np.allclose(np.hypot(dst[:, 0], dst[:, 1]), 12.0, rtol=1e-6)


@pytest.mark.parametrize("i", list(range(16)))
def test_batch_instance_ranges(i):
    w = workloads.batch_instance(i)
    assert w.seed == 1000 + i and 0 <= w.degree <= 3
    assert 128 <= w.n <= 1024
    g = w.geometry
    if i % 8 == 7:
        assert g.kind == "points" and 1e5 <= g.m <= 1e6
        assert np.allclose(np.hypot(g.src[:, 0], g.src[:, 1]), 0.75 * w.n, rtol=1e-5)
    else:
        assert g.kind in ("parallel", "fan")
        assert 180 <= g.n_view <= 1440 and g.n_det == int(round(1.5 * w.n))
        if g.kind == "fan":
            assert math.isclose(g.dso, 1000.0 * w.n / 512.0) and math.isclose(g.dod, 500.0 * w.n / 512.0)


def test_batch_instances_are_uneven():
    ws = [workloads.batch_instance(i) for i in range(16)]
    assert len({w.n for w in ws}) > 8
    assert {w.degree for w in ws} == {0, 1, 2, 3}
    assert {w.geometry.kind for w in ws} == {"parallel", "fan", "points"}


def test_transmission_data_scale_and_noise():
    rng = np.random.default_rng(0)
    e = rng.uniform(0.0, 40.0, 5000)
    y, kappa = workloads.transmission_data(e, seed=1, peak=3.0, I0=1e4)
    assert math.isclose(kappa * e.max(), 3.0)
    # Poisson noise on I0 exp(-3) ~ 500 counts: a few per cent of the line integral
    assert np.median(np.abs(y - e)) < 0.05 * e.max()
    y_hi, _ = workloads.transmission_data(e, seed=1, peak=3.0, I0=1e12)
    assert np.max(np.abs(y_hi - e)) < 1e-3 * e.max()
    y2, _ = workloads.transmission_data(e, seed=1, peak=3.0, I0=1e4)
    assert np.array_equal(y, y2)


def test_warmstart_params_ranges():
    for seed in (2_000_000, 2_000_001, 1_000_000 + 17):
        params, I0 = workloads.warmstart_params(seed)
        assert 5 <= params.shape[0] <= 40 and params.shape[1] == 6
        assert 1e3 <= I0 <= 1e5
        s = 256 / 64.0
        assert np.all(np.hypot(params[:, 0], params[:, 1]) <= 24.0 * s)
        assert np.all((params[:, 2:4] >= 2.0 * s) & (params[:, 2:4] <= 16.0 * s))
        assert np.all((params[:, 4] >= 0.0) & (params[:, 4] < math.pi))
        assert np.all((params[:, 5] >= -0.5) & (params[:, 5] < 1.0))
