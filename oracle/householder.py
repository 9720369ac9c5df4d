"""Householder-QR least squares on the Vandermonde matrix (validator).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section III describes the comparison method of the paper (MATLAB's polyfit):
build the Vandermonde matrix V (V[i][j] = x_i^j), factor V = QR with
Householder reflections, and solve R p = Q^T Y.  The printed algebra is
garbled ("(Q Q^T) R p = Q^T Y", "p = (Q^T Y) \\ R"); the reading used here is
the textbook one: p = R^{-1} (Q^T Y).  This is a different algorithm from the
normal equations, so agreement with the oracle pins the oracle's definition
of the fit (not its arithmetic).  Coefficients are in ascending order
(a_0..a_m), like the paper's X.
"""
from __future__ import annotations

import numpy as np


def vandermonde(x, m: int) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    V = np.empty((x.size, m + 1))
    V[:, 0] = 1.0
    for j in range(1, m + 1):
        V[:, j] = V[:, j - 1] * x
    return V


def lstsq(x, y, m: int) -> np.ndarray:
    """Ascending coefficients minimising ||V p - y||_2 by Householder QR."""
    R = vandermonde(x, m)
    z = np.array(y, dtype=np.float64)
    n, N = R.shape
    if n < N:
        raise ValueError("need at least m+1 points")
    for k in range(N):
        col = R[k:, k]
        alpha = np.linalg.norm(col)
        if alpha == 0.0:
            raise np.linalg.LinAlgError("rank deficient Vandermonde matrix")
        # reflect col onto -sign(col[0]) * alpha * e_1 (no cancellation)
        sgn = 1.0 if col[0] >= 0 else -1.0
        v = col.copy()
        v[0] += sgn * alpha
        vnorm2 = float(v @ v)
        # apply H = I - 2 v v^T / (v^T v) to the trailing columns and to z
        R[k:, k:] -= np.outer(v, (2.0 / vnorm2) * (v @ R[k:, k:]))
        z[k:] -= v * (2.0 / vnorm2) * (v @ z[k:])
    # back substitution on the upper triangle: R[:N] p = (Q^T y)[:N]
    p = np.zeros(N)
    for i in range(N - 1, -1, -1):
        p[i] = (z[i] - R[i, i + 1:N] @ p[i + 1:]) / R[i, i]
    return p
