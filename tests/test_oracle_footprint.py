"""Pins of the oracle's B-spline and footprint phi_theta against values fixed
outside the oracle: textbook B-spline values, scipy's independent B-spline,
the printed degree-1 closed form (Sec. III.C), direct quadrature of the basis
function along the line (eq. xray), unit mass, and symmetries."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.interpolate import BSpline

import oracle


def scipy_bspline(n):
    """Centred B-spline of degree n from scipy (independent of the oracle)."""
    knots = np.arange(n + 2, dtype=float) - 0.5 * (n + 1)
    b = BSpline.basis_element(knots, extrapolate=False)

    def f(x):
        v = b(x)
        return 0.0 if np.isnan(v) else float(v)
    return f


# ---------------------------------------------------------------- B-spline
@pytest.mark.parametrize("n,x,val", [
    (0, 0.0, 1.0), (0, 0.5, 0.5), (0, -0.5, 0.5), (0, 0.7, 0.0),
    (1, 0.0, 1.0), (1, 0.5, 0.5), (1, 1.0, 0.0),
    (2, 0.0, 0.75), (2, 0.5, 0.5), (2, 1.0, 0.125), (2, 1.5, 0.0),
    (3, 0.0, 2.0 / 3.0), (3, 1.0, 1.0 / 6.0), (3, -1.0, 1.0 / 6.0), (3, 2.0, 0.0),
])
def test_bspline_textbook_values(n, x, val):
    assert oracle.bspline(n, x) == pytest.approx(val, abs=1e-15)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_bspline_matches_scipy_and_partition_of_unity(n):
    ref = scipy_bspline(n)
    rng = np.random.default_rng(7)
    for x in rng.uniform(-2.5, 2.5, 200):
        if n == 0 and abs(abs(x) - 0.5) < 1e-12:
            continue
        assert oracle.bspline(n, x) == pytest.approx(ref(x), abs=1e-14)
    for x in rng.uniform(0, 1, 50):
        s = sum(oracle.bspline(n, x - k) for k in range(-4, 5))
        assert s == pytest.approx(1.0, abs=1e-14)


# ---------------------------------------------------------------- footprint
def line_quadrature(n, theta, y):
    """phi_theta(y) = int beta(t c + y s) beta(t s - y c) dt (eq. xray with
    theta^perp = (sin, -cos)), by adaptive quadrature with scipy's B-spline."""
    bs = scipy_bspline(n)
    c, s = math.cos(theta), math.sin(theta)
    half = 0.5 * (n + 1)
    # parameter t where either factor crosses one of its knots
    pts = []
    for k in np.arange(-half, half + 1e-9, 1.0):
        if abs(c) > 1e-15:
            pts.append((k - y * s) / c)
        if abs(s) > 1e-15:
            pts.append((k + y * c) / s)
    lim = 2 * half + abs(y) + 1
    pts = sorted(p for p in pts if -lim < p < lim)
    tot = 0.0
    edges = [-lim] + pts + [lim]
    for a, b in zip(edges[:-1], edges[1:]):
        if b - a < 1e-300:
            continue
        v, _ = quad(lambda t: bs(t * c + y * s) * bs(t * s - y * c), a, b, epsabs=1e-15, epsrel=1e-13, limit=200)
        tot += v
    return tot


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_footprint_theta0_is_bspline(n):
    # Prop. 1 with a zero scale: the Dirac leaves the other atom, phi_0 = beta^n.
    ref = scipy_bspline(n)
    for y in np.linspace(-2.3, 2.3, 47):
        if n == 0 and abs(abs(y) - 0.5) < 1e-12:
            continue
        assert oracle.footprint(n, 0.0, y) == pytest.approx(ref(y), abs=1e-14)
        assert oracle.footprint(n, math.pi / 2, y) == pytest.approx(ref(y), abs=1e-7)


def test_footprint_degree0_is_chord_length():
    # For the pixel basis phi_theta(y) is the chord of the unit square:
    # 1/a on |y| <= (a-b)/2, then linear down to 0 at |y| = (a+b)/2.
    rng = np.random.default_rng(3)
    for theta in rng.uniform(0, 2 * math.pi, 40):
        a = max(abs(math.cos(theta)), abs(math.sin(theta)))
        b = min(abs(math.cos(theta)), abs(math.sin(theta)))
        for y in rng.uniform(-1.0, 1.0, 25):
            ay = abs(y)
            if ay <= 0.5 * (a - b):
                ref = 1.0 / a
            elif ay < 0.5 * (a + b):
                ref = (0.5 * (a + b) - ay) / (a * b)
            else:
                ref = 0.0
            assert oracle.footprint(0, theta, y) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def printed_degree1(theta, y):
    """The closed form printed in Sec. III.C for the tensor B-spline (the
    9-term sum of truncated cubics over 6 a1^2 a2^2), with a1 = |cos|,
    a2 = |sin|, a3 = 2a1 + a2, a4 = a1 + 2a2, a5 = 2a1 + 2a2 and y measured
    from the left end of the support.  Its weights are those of four boxes,
    i.e. the degree-1 spline."""
    a1, a2 = abs(math.cos(theta)), abs(math.sin(theta))
    a3, a4, a5 = 2 * a1 + a2, a1 + 2 * a2, 2 * a1 + 2 * a2
    Y = y + a5 / 2

    def p(t):
        return max(t, 0.0) ** 3
    s = (p(Y) - 2 * p(Y - a1) - 2 * p(Y - a2) + p(Y - 2 * a1) + 4 * p(Y - a1 - a2)
         + p(Y - 2 * a2) - 2 * p(Y - a3) - 2 * p(Y - a4) + p(Y - a5))
    return s / (6 * a1 * a1 * a2 * a2)


def test_footprint_degree1_matches_printed_closed_form():
    rng = np.random.default_rng(11)
    for theta in rng.uniform(0.25, 1.3, 30):
        w = oracle.support_halfwidth(1, theta)
        for y in rng.uniform(-w * 1.1, w * 1.1, 30):
            assert oracle.footprint(1, theta, y) == pytest.approx(printed_degree1(theta, y), abs=1e-11)


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("theta", [0.3, 1.0, math.pi / 4, 2.5, 1e-3, 1e-6, math.pi / 2 - 1e-4])
def test_footprint_matches_line_quadrature(n, theta):
    w = oracle.support_halfwidth(n, theta)
    for y in np.linspace(-w * 0.98, w * 0.98, 9) + 0.0123:
        assert oracle.footprint(n, theta, y) == pytest.approx(line_quadrature(n, theta, y), abs=2e-10)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_footprint_unit_mass_and_symmetries(n):
    rng = np.random.default_rng(5 + n)
    for theta in list(rng.uniform(0, 2 * math.pi, 8)) + [1e-5, math.pi / 4]:
        a = max(abs(math.cos(theta)), abs(math.sin(theta)))
        b = min(abs(math.cos(theta)), abs(math.sin(theta)))
        m = n + 1
        w = 0.5 * m * (a + b)
        # breakpoints of phi_theta: -w + p a + q b (p, q = 0..n+1)
        br = sorted({-w + p * a + q * b for p in range(m + 1) for q in range(m + 1)})
        tot = 0.0
        for lo, hi in zip(br[:-1], br[1:]):
            if hi - lo > 0:
                tot += quad(lambda t: oracle.footprint(n, theta, t), lo, hi, epsabs=1e-15, epsrel=1e-13)[0]
        assert tot == pytest.approx(1.0, abs=1e-11)
        for y in rng.uniform(-w, w, 12):
            v = oracle.footprint(n, theta, y)
            assert oracle.footprint(n, theta, -y) == pytest.approx(v, abs=1e-13)
            assert oracle.footprint(n, -theta, y) == pytest.approx(v, abs=1e-13)
            assert oracle.footprint(n, theta + math.pi, y) == pytest.approx(v, abs=1e-12)
            assert oracle.footprint(n, math.pi / 2 - theta, y) == pytest.approx(v, abs=1e-12)


def test_footprint_support():
    for n in range(4):
        for theta in (0.2, 0.9, 2.0):
            w = oracle.support_halfwidth(n, theta)
            assert w == pytest.approx(0.5 * (n + 1) * (abs(math.cos(theta)) + abs(math.sin(theta))))
            assert oracle.footprint(n, theta, w) == 0.0
            assert oracle.footprint(n, theta, -w - 1e-9) == 0.0
            assert oracle.footprint(n, theta, w * (1 - 1e-3)) > 0.0
