"""Pins of the FP64 CGLS oracle (the reconstruction step of Sec. V, conjugate
gradients on the normal equations) against results fixed outside its
recurrences: the least-squares solution from a dense QR-based solver, the
Krylov-subspace optimality of each iterate solved directly on an explicit
basis, and the monotone decrease of the residual norm."""
import numpy as np
import pytest

import oracle
from oracle.cgls import cgls


def _tiny_problem(seed=7):
    grid = oracle.Grid(6, 6, 1)
    th, y = oracle.lines_parallel(np.arange(12) * (np.pi / 12), 10, -5.0, 1.0)
    A = lambda x: oracle.forward(grid, x, th, y)
    AT = lambda p: oracle.adjoint(grid, p, th, y)
    n = grid.nx * grid.ny
    H = np.stack([A(np.eye(n)[i].reshape(6, 6)) for i in range(n)], axis=1)   # m x n
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(H.shape[0])
    return grid, A, AT, H, b


def test_dense_matrix_is_the_operator():
    grid, A, AT, H, b = _tiny_problem()
    x = np.random.default_rng(1).standard_normal(36)
    assert np.allclose(H @ x, A(x.reshape(6, 6)), rtol=0, atol=1e-12)
    assert np.allclose(H.T @ b, AT(b).ravel(), rtol=0, atol=1e-12)


def test_converges_to_least_squares_solution():
    grid, A, AT, H, b = _tiny_problem()
    x_ls = np.linalg.lstsq(H, b, rcond=None)[0]       # minimum-norm LS solution
    x, gam, _ = cgls(A, AT, b, np.zeros((6, 6)), 200)
    assert np.linalg.norm(x.ravel() - x_ls) <= 1e-7 * np.linalg.norm(x_ls)
    assert gam[-1] <= 1e-20 * gam[0]


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_iterate_is_krylov_minimiser(k):
    # x_k = argmin ||b - H x|| over span{g, M g, ..., M^{k-1} g}, g = H^T b, M = H^T H
    grid, A, AT, H, b = _tiny_problem()
    g = H.T @ b
    M = H.T @ H
    V = [g]
    for _ in range(k - 1):
        V.append(M @ V[-1])
    Q, _ = np.linalg.qr(np.stack(V, axis=1))
    coeff = np.linalg.lstsq(H @ Q, b, rcond=None)[0]
    x_ref = Q @ coeff
    _, _, kept = cgls(A, AT, b, np.zeros((6, 6)), k, keep=(k,))
    assert np.linalg.norm(kept[k].ravel() - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_residual_decreases_and_gamma_matches_definition():
    grid, A, AT, H, b = _tiny_problem()
    keep = tuple(range(0, 16))
    _, gam, kept = cgls(A, AT, b, np.zeros((6, 6)), 15, keep=keep)
    res = [np.linalg.norm(b - H @ kept[k].ravel()) for k in keep]
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(len(res) - 1))
    for k in keep:
        s = H.T @ (b - H @ kept[k].ravel())
        assert abs(gam[k] - s @ s) <= 1e-9 * gam[0]


def test_nonzero_start():
    grid, A, AT, H, b = _tiny_problem()
    x0 = np.random.default_rng(3).standard_normal((6, 6))
    x_ls = np.linalg.lstsq(H, b, rcond=None)[0]
    x, _, _ = cgls(A, AT, b, x0, 200)
    # the LS solution is unique up to the null space of H; compare residuals
    assert abs(np.linalg.norm(b - H @ x.ravel()) - np.linalg.norm(b - H @ x_ls)) <= 1e-9 * np.linalg.norm(b)
