"""Pins of the oracle's 3-direction box-spline (Sec. III.D) and its x-ray
transform against facts outside the oracle's code: partition of unity of the
integer shifts, values at the lattice, adaptive quadrature along the line,
the paper's closed form (eq. projbox, read with 0-indexed alpha, at the
mirrored angle, see below), unit mass, symmetries, and the projector built on
it (mass conservation, adjoint identity, line quadrature of the image).

Orientation: the paper's closed form takes the box widths from <theta, u_d>
(its Fourier slice along theta), while lines here are {t theta + y
theta^perp} with theta^perp = (sin, -cos) (eq. rayparam), so the widths are
|<theta^perp, u_d>| = |sin|, |cos|, |sin - cos|.  For theta in (0, pi/4) the
paper's widths sin, cos, sin + cos are those of the angle -theta here."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle


def test_box_lattice_values_and_partition_of_unity():
    assert oracle.box3(0.0, 0.0) == 1.0
    for v in [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1), (2, 0)]:
        assert oracle.box3(*v) == 0.0
    assert oracle.box3(0.5, 0.5) == pytest.approx(0.5)
    rng = np.random.default_rng(11)
    for x in rng.uniform(-3, 3, size=(40, 2)):
        s = sum(oracle.box3(x[0] - i, x[1] - j) for i in range(-5, 6) for j in range(-5, 6))
        assert s == pytest.approx(1.0, abs=1e-14)


def test_box_symmetry_and_support():
    rng = np.random.default_rng(12)
    for x in rng.uniform(-1.5, 1.5, size=(50, 2)):
        v = oracle.box3(*x)
        assert v == pytest.approx(oracle.box3(-x[0], -x[1]), abs=1e-15)
        assert v == pytest.approx(oracle.box3(x[1], x[0]), abs=1e-15)
        inside = abs(x[0]) < 1 and abs(x[1]) < 1 and abs(x[0] - x[1]) < 1
        assert (v > 0) == inside


def _pieces_quad(f, lo, hi, n=240):
    """Adaptive quadrature on n equal sub-intervals (none of which can hide a
    narrow bump from the sampler)."""
    e = np.linspace(lo, hi, n + 1)
    return sum(quad(f, e[i], e[i + 1], limit=100, epsabs=1e-14, epsrel=1e-12)[0] for i in range(n))


def _line_quad(theta, yt):
    c, s = math.cos(theta), math.sin(theta)
    return _pieces_quad(lambda t: oracle.box3(yt * s + t * c, -yt * c + t * s), -3.0, 3.0)


@pytest.mark.parametrize("theta", [0.0, 0.3, math.pi / 4, 1.0, 2.2, 3.0, -0.7])
def test_box_footprint_matches_line_quadrature(theta):
    w = oracle.support_halfwidth_box(theta)
    for yt in np.linspace(-w * 1.05, w * 1.05, 23):
        assert oracle.footprint_box(theta, yt) == pytest.approx(_line_quad(theta, yt), abs=1e-8)


def _paper_projbox(theta_p, y):
    """eq. projbox with 0-indexed alpha (eq. alpha) and prefactor 1/(alpha_1 alpha_3 alpha_5)."""
    s, c = math.sin(theta_p), math.cos(theta_p)
    al = [0.0, s, 2 * s + c, c, s + 2 * c, 2 * (s + c)]
    return sum((-1) ** n * max(y - al[n], 0.0) ** 2 for n in range(6)) / (al[1] * al[3] * al[5])


@pytest.mark.parametrize("theta_p", [0.1, 0.35, 0.6, 0.78])
def test_box_footprint_matches_paper_closed_form(theta_p):
    # support [0, 2(s + c)] in the paper's coordinate; ours is centred
    half = math.sin(theta_p) + math.cos(theta_p)
    assert oracle.support_halfwidth_box(-theta_p) == pytest.approx(half, abs=1e-15)
    for y in np.linspace(0, 2 * half, 31):
        assert oracle.footprint_box(-theta_p, y - half) == pytest.approx(_paper_projbox(theta_p, y), abs=1e-12)


def test_box_footprint_axis_is_triangle_and_mass_one():
    for yt in np.linspace(-1.2, 1.2, 25):
        assert oracle.footprint_box(0.0, yt) == pytest.approx(max(0.0, 1 - abs(yt)), abs=1e-15)
    for theta in [0.0, 0.2, 0.9, math.pi / 4, 2.5]:
        w = oracle.support_halfwidth_box(theta)
        mass = quad(lambda y: oracle.footprint_box(theta, y), -w, w, limit=200, epsabs=1e-13)[0]
        assert mass == pytest.approx(1.0, abs=1e-10)


def test_box_footprint_symmetries():
    rng = np.random.default_rng(13)
    for theta in rng.uniform(0, 2 * math.pi, 12):
        for yt in rng.uniform(-1.5, 1.5, 5):
            v = oracle.footprint_box(theta, yt)
            assert v == pytest.approx(oracle.footprint_box(theta, -yt), abs=1e-13)
            assert v == pytest.approx(oracle.footprint_box(theta + math.pi, yt), abs=1e-13)
            assert v == pytest.approx(oracle.footprint_box(math.pi / 2 - theta, yt), abs=1e-13)


def test_box_projector_against_image_quadrature_and_mass():
    grid = oracle.Grid(6, 5, 1, h=1.3, cx=0.2, cy=-0.4, basis=1)
    rng = np.random.default_rng(14)
    coef = rng.standard_normal((5, 6))
    x1 = grid.cx + (np.arange(6) - 2.5) * grid.h
    x2 = grid.cy + (np.arange(5) - 2.0) * grid.h

    def image(x, y):
        return sum(coef[j, i] * oracle.box3((x - x1[i]) / grid.h, (y - x2[j]) / grid.h)
                   for j in range(5) for i in range(6))

    for theta, y in [(0.4, 0.7), (1.9, -1.1), (math.pi / 2, 0.3), (2.8, 2.0)]:
        c, s = math.cos(theta), math.sin(theta)
        ref = _pieces_quad(lambda t: image(y * s + t * c, -y * c + t * s), -12, 12, n=960)
        got = oracle.forward(grid, coef, np.array([theta]), np.array([y]))[0]
        assert got == pytest.approx(ref, abs=1e-8)
    # mass: int P_theta(y) dy = h^2 sum c, with a fine detector
    for theta in [0.3, 1.2]:
        ys = np.arange(-12, 12, 1 / 256.0)
        p = oracle.forward(grid, coef, np.full(ys.size, theta), ys)
        assert p.sum() / 256.0 == pytest.approx(grid.h ** 2 * coef.sum(), abs=2e-7)


def test_box_projector_adjoint_identity_and_enumeration():
    grid = oracle.Grid(9, 8, 1, basis=1)
    rng = np.random.default_rng(15)
    th, y = oracle.lines_parallel(np.linspace(0, math.pi, 23, endpoint=False), 15, -7.3, 1.0)
    c = rng.standard_normal((8, 9))
    p = rng.standard_normal(th.size)
    lhs = float(oracle.forward(grid, c, th, y) @ p)
    rhs = float((c * oracle.adjoint(grid, p, th, y)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.array_equal(oracle.forward(grid, c, th, y, brute=True), oracle.forward(grid, c, th, y))
