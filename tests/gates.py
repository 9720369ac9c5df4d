"""Tolerances of the GPU parity tests, in one place.

Forward error.  The coefficients are compared with the oracle's FP64 fit of
the same stored points, in the mapped basis (normwise relative error of Xt).
The stated bounds are 1e-6 for FP64 accumulation and 1e-5 for
compensated FP32 of degree <= 3 on [-1, 1].  Beyond that, a coefficient is
only as well determined as the normal system allows: to first order its
error is cond(A) times the relative perturbation of A and B.  So a forward
gate is used where it means something, and nowhere else:
  * ``forward_gate`` returns max(base, cond(A) * eps * 4m) while that stays at
    or below 1e-3 (eps: 2^-53 for FP64 sums, 2^-24 for FP32 powers; 4m
    covers the roundings of a power t^k, k <= 2m, and its product with y);
  * above 1e-3 the forward error is reported and not gated (the data leave
    the coefficients undetermined at that level).

Backward error.  Every ok result is also held to a gate that does not depend
on cond(A): the normwise backward error of the GPU's Xt in the oracle's own
normal equations A Xt = B (Rigal and Gaches),
    eta = |A Xt - B| / (|A| |Xt| + |B|)           (2-norms),
is the smallest relative perturbation of A and B for which Xt is the exact
solution.  A solve in FP64 from sums that carry a relative error delta gives
eta of about delta, whatever cond(A) is, so a dropped term, a wrong index or
a wrong sign shows up as eta of order one.  ``backward_gate`` gives the
bound per accumulation: compensated FP32 sums are exact up to the roundings
of the per-point powers (at most (3k + 16) * 2^-24 of sum |t|^k, with |t| <= 1
after the map), FP64 ones up to the FP64 roundings of a lane's share.  The
oracle's own sums are sequential FP64 sums of n terms, good to
(n - 1) 2^-53 of the sum of their magnitudes, so the FP64 gate adds
2 n 2^-53 to its floor of 1e-12 (for BF16 data, whose repeated values make
the rounding errors of both sides systematic, this term is what is seen).

Saved sums.  ``sums_bound`` is the error bound of one power sum of the
compensated FP32 path: t = (x - c) s carries two FP32 roundings, t^k by the
running product k - 1 more (so 3k - 1 in all), the product with y one more,
and the plain FP32 batch that precedes each TwoSum fold at most B - 1 more,
B the points of a batch per packed lane (8 single-series at degree <= 6,
16 above; 16 in the batched stage rings).  The folds, the double-float
trees and the FP64 combine add terms of order 2^-48.
"""
import numpy as np

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -53

FORWARD_CEILING = 1e-3

# normwise backward error of Xt in the oracle's normal equations
BACKWARD = {"comp": 1e-5, "f64": 1e-12, "naive": 1e-3}


def hankel(S, m):
    return np.array([[S[j + k] for k in range(m + 1)] for j in range(m + 1)], dtype=np.float64)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def forward_gate(accum, m, cond, base=None):
    """Gate on the normwise relative error of Xt, or None (reported only).
    base: the floor of the gate (1e-6 FP64, 1e-5 FP32 unless given)."""
    if accum == "f64":
        tol = max(1e-6 if base is None else base, cond * EPS64 * 4 * m)
    else:
        tol = max(1e-5 if base is None else base, cond * EPS32 * 4 * m)
    return tol if tol <= FORWARD_CEILING else None


def backward_error(A, B, Xt):
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Xt = np.asarray(Xt, dtype=np.float64)
    r = A @ Xt - B
    return float(np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(Xt) + np.linalg.norm(B)))


def backward_gate(accum, n=0):
    """Gate on the backward error for n summed points."""
    if accum == "f64":
        return BACKWARD["f64"] + 2.0 * n * EPS64
    return BACKWARD[accum]


def sums_bound(k, scale, batch=16):
    """Error bound of a compensated FP32 power sum of degree k (S_k) or of a
    right-hand side T_{k} (pass k + 1 for the product with y), relative to
    scale = sum_i |t_i|^k (or sum_i |t_i|^k |y_i|)."""
    return (3 * k + batch) * EPS32 * scale


def sums_bound_for(accum, k, scale, lane_terms):
    """As sums_bound for any accumulation.  Naive FP32 sums a lane's whole share
    (lane_terms points, at most ceil(n / 32)) before the exact double-float
    trees; FP64 accumulation rounds once per point of a lane's share plus the
    tree and chunk-combine additions (64 covers those)."""
    if accum == "comp":
        return sums_bound(k, scale, batch=16)
    if accum == "naive":
        return (3 * k + lane_terms + 16) * EPS32 * scale
    return (3 * k + lane_terms + 64) * EPS64 * scale


def check_coefficients(Xt, ref_Xt, A, B, accum, m, base=None, n=0):
    """Forward gate where it applies, backward gate always (n: points summed).
    Returns (forward error, forward gate or None, backward error)."""
    cond = float(np.linalg.cond(A))
    ef = rel(Xt, ref_Xt)
    tol = forward_gate(accum, m, cond, base)
    eta = backward_error(A, B, Xt)
    if tol is not None:
        assert ef <= tol, ("forward", ef, tol, m, cond)
    assert eta <= backward_gate(accum, n), ("backward", eta, backward_gate(accum, n), m, cond)
    return ef, tol, eta
