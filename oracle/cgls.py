"""FP64 conjugate gradients on the normal equations (CGLS), written plainly.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``): only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.

Sec. V reconstructs by solving the normal equations A^T A x = A^T y with
conjugate gradients (the paper does not fix the variant).  This is the
Hestenes-Stiefel recurrence applied to the normal equations without forming
A^T A: with x_0 given,

    r_0 = b - A x_0,  s_0 = A^T r_0,  p_0 = s_0,  gamma_0 = <s_0, s_0>
    q_k = A p_k,  alpha_k = gamma_k / <q_k, q_k>
    x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k q_k
    s_{k+1} = A^T r_{k+1},  gamma_{k+1} = <s_{k+1}, s_{k+1}>
    p_{k+1} = s_{k+1} + (gamma_{k+1} / gamma_k) p_k

x_k minimises ||b - A x|| over x_0 + K_k(A^T A, A^T r_0).  ``A`` and ``AT``
are callables (for the projector: :func:`oracle.forward` and
:func:`oracle.adjoint` on one grid and line list).
"""
from __future__ import annotations

import numpy as np


def cgls(A, AT, b, x0, iters: int, keep=()):
    """Run ``iters`` iterations.  Returns (x_iters, gammas, kept) with gammas
    the list gamma_0..gamma_iters and kept a dict {k: x_k} for k in ``keep``."""
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A(x)
    s = AT(r)
    p = s.copy()
    gamma = float(np.dot(s.ravel(), s.ravel()))
    gammas = [gamma]
    kept = {0: x.copy()} if 0 in keep else {}
    for k in range(1, iters + 1):
        q = A(p)
        qq = float(np.dot(q.ravel(), q.ravel()))
        alpha = gamma / qq if qq > 0.0 else 0.0
        x = x + alpha * p
        r = r - alpha * q
        s = AT(r)
        gamma_new = float(np.dot(s.ravel(), s.ravel()))
        beta = gamma_new / gamma if gamma > 0.0 else 0.0
        p = s + beta * p
        gamma = gamma_new
        gammas.append(gamma)
        if k in keep:
            kept[k] = x.copy()
    return x, gammas, kept
