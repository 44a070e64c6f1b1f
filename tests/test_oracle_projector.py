"""Pins of the oracle's projector and adjoint against mathematics outside it:
direct line quadrature of the spline image (eq. xray with eq. def_f), Siddon's
intersection lengths at degree 0 (Sec. II.A), conservation of mass, the
theta -> theta + pi symmetry, the adjoint identity, Lemma 1 through
Algorithm 2's candidate set, and the enumeration of the nonzero pairs."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.interpolate import BSpline

import oracle
import workloads


def scipy_bspline(n):
    knots = np.arange(n + 2, dtype=float) - 0.5 * (n + 1)
    b = BSpline.basis_element(knots, extrapolate=False)
    return lambda x: np.nan_to_num(b(x))


def node_coords(nx, ny, h, cx, cy):
    return cx + (np.arange(nx) - 0.5 * (nx - 1)) * h, cy + (np.arange(ny) - 0.5 * (ny - 1)) * h


def image_line_integral(coef, n, h, cx, cy, theta, y):
    """int f(t theta + y theta^perp) dt with f = sum c_k beta((x1-x1k)/h) beta((x2-x2k)/h),
    by adaptive quadrature split at every knot crossing."""
    ny, nx = coef.shape
    x1, x2 = node_coords(nx, ny, h, cx, cy)
    bs = scipy_bspline(n)
    c, s = math.cos(theta), math.sin(theta)
    px, py = y * s, -y * c
    half = 0.5 * (n + 1) * h

    def f(t):
        X, Y = px + t * c, py + t * s
        return float(bs((X - x1) / h) @ coef.T @ bs((Y - x2) / h)) if False else \
            float(np.sum(coef * np.outer(bs((Y - x2) / h), bs((X - x1) / h))))
    # knots along x1: x1k + (q - (n+1)/2) h; along x2 likewise
    pts = []
    kn1 = np.unique(np.concatenate([x1 + (q - 0.5 * (n + 1)) * h for q in range(n + 2)]))
    kn2 = np.unique(np.concatenate([x2 + (q - 0.5 * (n + 1)) * h for q in range(n + 2)]))
    if abs(c) > 1e-14:
        pts += list((kn1 - px) / c)
    if abs(s) > 1e-14:
        pts += list((kn2 - py) / s)
    R = math.hypot(nx, ny) * h + 4 * half + abs(y)
    pts = sorted(p for p in pts if -R < p < R)
    edges = [-R] + pts + [R]
    tot = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        if b - a > 1e-12:
            tot += quad(f, a, b, epsabs=1e-13, epsrel=1e-12, limit=100)[0]
    return tot


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_forward_matches_line_quadrature(n):
    rng = np.random.default_rng(100 + n)
    nx, ny, h, cx, cy = 5, 4, 0.7, 0.3, -0.2
    g = oracle.Grid(nx, ny, n, h, cx, cy)
    coef = rng.uniform(-1, 1, (ny, nx))
    th = rng.uniform(0, 2 * math.pi, 6)
    yy = rng.uniform(-2.0, 2.0, 6)
    got = oracle.forward(g, coef, th, yy, brute=True)
    for k in range(th.size):
        ref = image_line_integral(coef, n, h, cx, cy, th[k], yy[k])
        assert got[k] == pytest.approx(ref, abs=1e-9 * max(1.0, abs(ref)))


def test_degree0_reduces_to_siddon():
    # Sec. II.B: with the pixel basis, Algorithm 2 reduces to Siddon's method.
    rng = np.random.default_rng(21)
    g = oracle.Grid(16, 12, 0, 1.3, 0.4, -0.9)
    coef = rng.uniform(-1, 2, (12, 16))
    th = rng.uniform(0, 2 * math.pi, 60)
    yy = rng.uniform(-12, 12, 60)
    got = oracle.forward(g, coef, th, yy, brute=True)
    for k in range(60):
        assert got[k] == pytest.approx(oracle.siddon_line(g, coef, th[k], yy[k]), abs=1e-11)


def projection_breakpoints(g, theta):
    """Offsets y at which P_theta(y) changes polynomial piece: for every node,
    its offset plus the breakpoints -w + p a + q b of phi_theta (scaled by h)."""
    n = g.degree
    c, s = math.cos(theta), math.sin(theta)
    a, b = max(abs(c), abs(s)), min(abs(c), abs(s))
    m = n + 1
    w = 0.5 * m * (a + b)
    x1, x2 = node_coords(g.nx, g.ny, g.h, g.cx, g.cy)
    X1, X2 = np.meshgrid(x1, x2)
    yk = (X1 * s - X2 * c).ravel()
    off = np.array([(-w + p * a + q * b) * g.h for p in range(m + 1) for q in range(m + 1)])
    return np.unique((yk[:, None] + off[None, :]).ravel())


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_mass_conservation(n):
    # int P_theta(y) dy = h^2 sum_k c_k for every theta (unit mass of phi_theta).
    rng = np.random.default_rng(40 + n)
    g = oracle.Grid(6, 5, n, 0.8, 0.1, 0.2)
    coef = rng.uniform(-1, 1, (5, 6))
    xg, wg = np.polynomial.legendre.leggauss(4)  # exact to degree 7 >= 2n+1
    for theta in (0.0, 0.37, 1.1, math.pi / 4, 2.9):
        br = projection_breakpoints(g, theta)
        lo, hi = br[:-1], br[1:]
        keep = hi - lo > 1e-12
        lo, hi = lo[keep], hi[keep]
        mid, hw = 0.5 * (lo + hi), 0.5 * (hi - lo)
        ys = (mid[:, None] + hw[:, None] * xg[None, :]).ravel()
        P = oracle.forward(g, coef, np.full(ys.size, theta), ys, brute=True).reshape(-1, 4)
        tot = float(np.sum(hw * (P @ wg)))
        assert tot == pytest.approx(g.h ** 2 * coef.sum(), abs=1e-11)


def test_theta_plus_pi_symmetry():
    # The line (theta + pi, -y) is the line (theta, y) with the opposite direction.
    rng = np.random.default_rng(9)
    for n in range(4):
        g = oracle.Grid(9, 7, n, 1.0, 0.0, 0.0)
        coef = rng.uniform(-1, 1, (7, 9))
        th = rng.uniform(0, math.pi, 30)
        yy = rng.uniform(-5, 5, 30)
        a = oracle.forward(g, coef, th, yy, brute=True)
        b = oracle.forward(g, coef, th + math.pi, -yy, brute=True)
        np.testing.assert_allclose(a, b, atol=1e-12)


def test_adjoint_identity():
    rng = np.random.default_rng(13)
    for n in range(4):
        g = oracle.Grid(10, 8, n, 0.9, 0.2, 0.1)
        x = rng.uniform(-1, 1, (8, 10))
        th = rng.uniform(0, 2 * math.pi, 70)
        yy = rng.uniform(-6, 6, 70)
        p = rng.uniform(-1, 1, 70)
        Ax = oracle.forward(g, x, th, yy)
        Atp = oracle.adjoint(g, p, th, yy)
        lhs, rhs = float(Ax @ p), float(np.sum(x * Atp))
        assert lhs == pytest.approx(rhs, abs=1e-12 * np.linalg.norm(Ax) * np.linalg.norm(p))
        # and a transposition of the image axes is caught: the matrix is not symmetric in (i, j)
        assert abs(float(np.sum(x.T[:8, :8] * Atp[:8, :8])) - rhs) > 1e-6


def test_row_enumeration_equals_brute_force():
    rng = np.random.default_rng(17)
    for n in range(4):
        g = oracle.Grid(24, 20, n, 1.0, 0.5, -0.25)
        coef = rng.uniform(-1, 1, (20, 24))
        th = np.concatenate([rng.uniform(0, 2 * math.pi, 40), [0.0, math.pi / 2, math.pi / 4, 1e-7]])
        yy = rng.uniform(-14, 14, th.size)
        a = oracle.forward(g, coef, th, yy, brute=True)
        b = oracle.forward(g, coef, th, yy, brute=False)
        assert np.array_equal(a, b)
        ca, _, oa, ia = oracle.visited(g, th, yy, brute=True, with_index=True)
        cb, _, ob, ib = oracle.visited(g, th, yy, brute=False, with_index=True)
        assert np.array_equal(ca, cb) and np.array_equal(ia, ib)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_algorithm2_with_K_equal_n_covers_every_pair(n):
    # Lemma 1: the tensor beta^n support lies in a disk of radius (n+1)/sqrt 2,
    # so K = ceil(sqrt 2 R - 1) = n neighbours suffice.
    rng = np.random.default_rng(60 + n)
    g = oracle.Grid(20, 20, n, 1.0, 0.0, 0.0)
    coef = rng.uniform(-1, 1, (20, 20))
    th = rng.uniform(0, 2 * math.pi, 150)
    yy = rng.uniform(-13, 13, 150)
    counts, _, offs, idx = oracle.visited(g, th, yy, with_index=True)
    ref = oracle.forward(g, coef, th, yy)
    missed_with_fewer = 0
    for r in range(th.size):
        nz = set(idx[offs[r]:offs[r + 1]].tolist())
        cand, val = oracle.alg2_line(g, coef, th[r], yy[r], n)
        assert nz <= set(cand.tolist())
        assert val == pytest.approx(ref[r], abs=1e-12)
        if n > 0:
            cand2, _ = oracle.alg2_line(g, coef, th[r], yy[r], n - 1)
            missed_with_fewer += not nz <= set(cand2.tolist())
    if n > 0:
        assert missed_with_fewer > 0   # K = n is also necessary


def test_parallel64_linear_visited_set_margin():
    # The nonzero set is decided by |y~| < w; on this workload no pair lies
    # within 1e-5 of the boundary, so float32 and float64 decisions agree.
    wl = workloads.workload("parallel64_linear")
    g = oracle.Grid(wl.n, wl.n, wl.degree, wl.h)
    geo = wl.geometry
    th, yy = oracle.lines_parallel(geo.view_angle.astype(np.float64), geo.n_det, geo.det0, geo.ddet)
    counts, gap = oracle.visited(g, th, yy, brute=True)
    assert gap > 1e-5
    assert counts.sum() > 0


def test_fan_and_points_geometry():
    # A fan line passes through its source and its bin centre.
    beta = np.array([0.0, 0.7, 2.0, 4.5], dtype=np.float32)
    th, yy = oracle.lines_fan(beta, 100.0, 50.0, 5, -2.0, 1.0)
    for v, b in enumerate(beta.astype(np.float64)):
        S = 100.0 * np.array([math.cos(b), math.sin(b)])
        u = np.array([-math.sin(b), math.cos(b)])
        for j in range(5):
            D = -50.0 * np.array([math.cos(b), math.sin(b)]) + (-2.0 + j) * u
            r = v * 5 + j
            perp = np.array([math.sin(th[r]), -math.cos(th[r])])
            assert S @ perp == pytest.approx(yy[r], abs=1e-10)
            assert D @ perp == pytest.approx(yy[r], abs=1e-10)
            d = (D - S) / np.linalg.norm(D - S)
            assert d @ np.array([math.cos(th[r]), math.sin(th[r])]) == pytest.approx(1.0, abs=1e-12)
    src, dst = workloads.random_lines_circle(20, 10.0, 3)
    th, yy = oracle.lines_points(src, dst)
    for r in range(20):
        perp = np.array([math.sin(th[r]), -math.cos(th[r])])
        assert src[r].astype(float) @ perp == pytest.approx(yy[r], abs=1e-9)
        assert dst[r].astype(float) @ perp == pytest.approx(yy[r], abs=1e-9)
