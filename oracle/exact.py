"""Exact rational restatement of the fit of Section II (tiny inputs only).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Inputs are taken as exact rationals (``fractions.Fraction`` of their decimal
strings or of the FP64 values), so the power sums S_k, T_k, the Hankel system
A[j][k] = S_{j+k}, B[j] = T_j and its solution are exact.  Elimination needs
no pivoting rule in exact arithmetic beyond skipping zero pivots.  Pure-Python
loops: keep n and m small.
"""
from __future__ import annotations

from fractions import Fraction


def as_fraction(v) -> Fraction:
    if isinstance(v, Fraction):
        return v
    if isinstance(v, str):
        return Fraction(v)
    return Fraction(float(v))  # exact value of the binary double


def powersums(x, y, m: int):
    xs = [as_fraction(v) for v in x]
    ys = [as_fraction(v) for v in y]
    S = [sum((xi ** k for xi in xs), Fraction(0)) for k in range(2 * m + 1)]
    T = [sum((xi ** k * yi for xi, yi in zip(xs, ys)), Fraction(0)) for k in range(m + 1)]
    return S, T


def solve(S, T, m: int):
    """Exact solution of A X = B with A[j][k] = S[j+k], B[j] = T[j].

    Returns None when A is singular."""
    N = m + 1
    A = [[S[j + k] for k in range(N)] + [T[j]] for j in range(N)]
    for col in range(N):
        piv = next((r for r in range(col, N) if A[r][col] != 0), None)
        if piv is None:
            return None
        A[col], A[piv] = A[piv], A[col]
        for r in range(col + 1, N):
            f = A[r][col] / A[col][col]
            A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    X = [Fraction(0)] * N
    for i in range(N - 1, -1, -1):
        acc = A[i][N] - sum((A[i][j] * X[j] for j in range(i + 1, N)), Fraction(0))
        X[i] = acc / A[i][i]
    return X


def fit(x, y, m: int):
    S, T = powersums(x, y, m)
    return solve(S, T, m), S, T


def sse(X, x, y) -> Fraction:
    tot = Fraction(0)
    for xi, yi in zip(x, y):
        xi = as_fraction(xi)
        yi = as_fraction(yi)
        f = sum((as_fraction(a) * xi ** j for j, a in enumerate(X)), Fraction(0))
        tot += (yi - f) ** 2
    return tot
