"""Pins of the CPU oracle to facts the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a printed
value of the paper, a closed form, exact rational arithmetic, a different
algorithm (Householder QR, LAPACK, torch autograd, finite differences) or a
brute-force integer sum.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import exact, householder
from tests.conftest import read_golden

EPS = np.finfo(np.float64).eps


def _table1():
    rows, _ = read_golden("table1_sample.txt")
    xs = [r[0] for r in rows]
    ys = [r[1] for r in rows]
    return xs, ys, np.array([float(v) for v in xs]), np.array([float(v) for v in ys])


def _hankel(S, m):
    return np.array([[S[j + k] for k in range(m + 1)] for j in range(m + 1)])


# --- Section III, Tables II-IV: the polyfit column is the exact LSE minimiser ----------

@pytest.mark.parametrize("m", [1, 2, 3])
def test_tables_2_to_4_polyfit_coefficients(m):
    _, _, x, y = _table1()
    rows, _ = read_golden("tables2_4_polyfit.txt")
    row = next(r for r in rows if int(r[0]) == m)
    printed = row[1:]
    out = oracle.fit(x, y, m)
    assert out["status"] == "ok"
    assert len(printed) == m + 1
    for v, s in zip(out["X"], printed):
        decimals = len(s.split(".")[1])
        assert round(float(v), decimals) == float(s), (out["X"], printed)


def test_table5_fitted_values_and_sse():
    _, _, x, y = _table1()
    rows, _ = read_golden("table5_fitted.txt")
    yp = np.array([float(r[2]) for r in rows if len(r) == 3])
    sse_f = float(next(r[1] for r in rows if r[0] == "sse_f"))
    sse_p = float(next(r[1] for r in rows if r[0] == "sse_p"))
    polyfit_rounded = [-4.7551, 17.5109, 0.1086, -0.0016]  # Table IV, polyfit column
    # y_p of Table V is f_p evaluated with the printed polyfit coefficients
    f = oracle.evaluate(polyfit_rounded, x)
    assert np.all(np.abs(f - yp) <= 1e-4 + 1e-7 * np.abs(yp)), (f, yp)
    assert abs(oracle.sse(polyfit_rounded, x, y) - sse_p) <= 1e-3
    # the exact minimiser cannot do worse than any printed fit, and sits close to the
    # paper's own m = 3 fit
    out = oracle.fit(x, y, 3)
    s_min = oracle.sse(out["X"], x, y)
    assert s_min <= sse_f <= sse_p
    assert sse_f - s_min < 1e-3
    # stationarity: nudging any coefficient raises the SSE
    for j in range(4):
        for d in (1e-4, -1e-4):
            Xd = out["X"].copy()
            Xd[j] += d * max(1.0, abs(Xd[j]))
            assert oracle.sse(Xd, x, y) > s_min


# --- exact rationals -----------------------------------------------------------------

def _sum_bound(terms, n, k):
    return (n + 2) * (k + 2) * EPS * float(np.sum(np.abs(terms)))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_exact_rational_table1(m):
    _, _, x, y = _table1()
    Xq, Sq, Tq = exact.fit(list(x), list(y), m)  # exact values of the FP64 inputs
    out = oracle.fit(x, y, m)
    for k in range(2 * m + 1):
        assert abs(out["S"][k] - float(Sq[k])) <= _sum_bound(x ** k, x.size, k)
    for k in range(m + 1):
        assert abs(out["T"][k] - float(Tq[k])) <= _sum_bound(x ** k * y, x.size, k)
    cond = np.linalg.cond(_hankel(out["S"], m))
    Xe = np.array([float(v) for v in Xq])
    rel = np.linalg.norm(out["X"] - Xe) / np.linalg.norm(Xe)
    assert rel <= 1e3 * cond * EPS, (rel, cond)


@pytest.mark.parametrize("seed", range(6))
def test_exact_rational_random_tiny(seed):
    rng = np.random.default_rng(100 + seed)
    m = 1 + seed % 4
    n = m + 1 + int(rng.integers(0, 12))
    x = rng.uniform(-2.0, 3.0, n)
    y = rng.normal(0.0, 2.0, n)
    Xq, Sq, Tq = exact.fit(list(x), list(y), m)
    out = oracle.fit(x, y, m)
    assert out["status"] == "ok"
    cond = np.linalg.cond(_hankel(out["S"], m))
    Xe = np.array([float(v) for v in Xq])
    rel = np.linalg.norm(out["X"] - Xe) / np.linalg.norm(Xe)
    assert rel <= 1e3 * cond * EPS, (rel, cond)


# --- closed form of the straight line (Section II, f(x) = a + bx) ----------------------

@pytest.mark.parametrize("seed", range(4))
def test_closed_form_line(seed):
    rng = np.random.default_rng(200 + seed)
    n = 50 + 37 * seed
    x = rng.uniform(-5.0, 20.0, n)
    y = 3.0 - 1.25 * x + rng.normal(0.0, 0.5, n)
    q = [Fraction(float(v)) for v in x]
    r = [Fraction(float(v)) for v in y]
    sx, sy = sum(q), sum(r)
    sxx = sum(a * a for a in q)
    sxy = sum(a * b for a, b in zip(q, r))
    b = (n * sxy - sx * sy) / (n * sxx - sx * sx)
    a = (sy - b * sx) / n
    out = oracle.fit(x, y, 1)
    assert out["status"] == "ok"
    np.testing.assert_allclose(out["X"], [float(a), float(b)], rtol=1e-11, atol=1e-12)


# --- noiseless data: the fit recovers the generating polynomial ---------------------------

@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_noiseless_recovery(m):
    rng = np.random.default_rng(300 + m)
    coef = rng.integers(-5, 6, m + 1).astype(np.float64)
    coef[-1] = coef[-1] or 2.0
    x = np.linspace(-1.5, 2.0, 40 + 3 * m)
    y = np.zeros_like(x)
    for k in range(m, -1, -1):
        y = y * x + coef[k]
    out = oracle.fit(x, y, m)
    assert out["status"] == "ok"
    cond = np.linalg.cond(_hankel(out["S"], m))
    assert np.linalg.norm(out["X"] - coef) <= 1e2 * cond * EPS * np.linalg.norm(coef)
    # in exact arithmetic the recovery is exact
    if m <= 3:
        Xq, _, _ = exact.fit(list(x), list(y), m)
        yq = [Fraction(float(v)) for v in y]
        # y was rounded to doubles; the exact fit of those doubles is within rounding of coef
        assert all(abs(float(v) - c) < 1e-9 for v, c in zip(Xq, coef))
        del yq
    # a fit of higher degree than the data keeps the top coefficients at zero
    out2 = oracle.fit(x, y, m + 1)
    assert abs(out2["X"][-1]) < 1e-7


# --- independent algorithm: Householder QR on the Vandermonde matrix (Section III) ---------

@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
def test_householder_qr_agreement_mapped(m):
    d = synth.small_series(2000, seed=400 + m, lo=-1.0, hi=1.0, m=m, noise=0.05,
                           dtype=np.float64)
    out = oracle.fit(d["x"], d["y"], m)
    p = householder.lstsq(d["x"], d["y"], m)
    cond = np.linalg.cond(_hankel(out["S"], m))
    rel = np.linalg.norm(out["X"] - p) / np.linalg.norm(p)
    assert rel <= 1e2 * cond * EPS, (rel, cond)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_householder_qr_agreement_table1(m):
    _, _, x, y = _table1()
    out = oracle.fit(x, y, m)
    p = householder.lstsq(x, y, m)
    cond = np.linalg.cond(_hankel(out["S"], m))
    assert np.linalg.norm(out["X"] - p) / np.linalg.norm(p) <= 1e2 * cond * EPS


def test_householder_itself_against_lapack():
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, 300)
    y = rng.normal(size=300)
    V = householder.vandermonde(x, 4)
    ref = np.linalg.lstsq(V, y, rcond=None)[0]
    np.testing.assert_allclose(householder.lstsq(x, y, 4), ref, rtol=1e-10, atol=1e-12)


# --- residual orthogonality V^T r = 0 ---------------------------------------------------

@pytest.mark.parametrize("m", [1, 3, 5, 8])
def test_residual_orthogonality(m):
    d = synth.small_series(5000, seed=500 + m, m=m, noise=0.1, dtype=np.float64)
    out = oracle.fit(d["x"], d["y"], m)
    r = d["y"] - oracle.evaluate(out["X"], d["x"])
    cond = np.linalg.cond(_hankel(out["S"], m))
    for k in range(m + 1):
        xk = d["x"] ** k
        assert abs(np.sum(xk * r)) <= 10 * cond * EPS * np.sum(np.abs(xk) * (np.abs(r) + np.abs(d["y"])))


# --- power sums: bit-exact against integer sums -----------------------------------------

@pytest.mark.parametrize("m", [1, 2, 3])
def test_powersums_bit_exact_int64(m):
    rng = np.random.default_rng(600 + m)
    n = 3001
    xi = rng.integers(-8, 9, n)
    yi = rng.integers(-100, 101, n)
    S, T = oracle.powersums(xi.astype(np.float64), yi.astype(np.float64), m)
    for k in range(2 * m + 1):
        assert S[k] == float(int(np.sum(xi.astype(np.int64) ** k)))
    for k in range(m + 1):
        assert T[k] == float(int(np.sum(xi.astype(np.int64) ** k * yi)))


def test_normal_matrix_equals_vandermonde_gram():
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, 777)
    y = rng.normal(size=777)
    m = 4
    S, T = oracle.powersums(x, y, m)
    V = householder.vandermonde(x, m)
    np.testing.assert_allclose(_hankel(S, m), V.T @ V, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(T, V.T @ y, rtol=1e-12, atol=1e-10)


# --- Gaussian elimination with partial pivoting -------------------------------------------

@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_gauss_against_lapack(m):
    rng = np.random.default_rng(900 + m)
    x = rng.uniform(0.0, 10.0, 400)  # S_1 > S_0: pivoting is exercised
    y = rng.normal(size=400)
    S, T = oracle.powersums(x, y, m)
    st, X = oracle.solve(S, T, m)
    assert st == "ok"
    ref = np.linalg.solve(_hankel(S, m), T)
    cond = np.linalg.cond(_hankel(S, m))
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 1e2 * cond * EPS


def test_gauss_needs_pivoting():
    # leading entry tiny relative to the column: elimination without row exchange
    # would lose all accuracy; partial pivoting must not.
    x = np.array([1e3, 1e3 + 1, 1e3 + 2, 1e3 + 3.5, 1e3 + 5])
    y = np.array([1.0, 3.0, 2.0, 5.0, 4.0])
    S, T = oracle.powersums(x, y, 1)
    st, X = oracle.solve(S, T, 1)
    Xq, _, _ = exact.fit(list(x), list(y), 1)
    assert st == "ok"
    np.testing.assert_allclose(X, [float(v) for v in Xq], rtol=1e-9)


# --- statuses --------------------------------------------------------------------------

def test_status_cases():
    assert oracle.fit([1.0, 2.0], [1.0, 2.0], 2)["status"] == "n_too_small"
    assert oracle.fit([2.0] * 10, list(range(10)), 1)["status"] == "singular"
    assert oracle.fit([1.0, 2.0, 2.0, 1.0], [1.0, 2.0, 3.0, 4.0], 2)["status"] == "singular"
    assert oracle.fit([1.0, 2.0, 3.0], [1.0, np.nan, 3.0], 1)["status"] == "nonfinite"
    assert oracle.fit([1.0, np.inf, 3.0], [1.0, 2.0, 3.0], 1)["status"] == "nonfinite"
    assert oracle.map_constants(1.0, 1.0, True)[0] == "bad_interval"
    assert oracle.map_constants(2.0, 1.0, False)[0] == "bad_interval"
    assert oracle.map_constants(0.0, np.inf, False)[0] == "bad_interval"
    out = oracle.fit([1.0, 2.0], [1.0, 2.0], 2)
    assert np.all(np.isnan(out["X"]))
    # the paper's n >= 2 is enough for a line
    out = oracle.fit([1.0, 2.0], [3.0, 5.0], 1)
    assert out["status"] == "ok"
    np.testing.assert_allclose(out["X"], [1.0, 2.0], rtol=1e-14)


# --- affine map and un-map -------------------------------------------------------------

def test_map_constants_and_range():
    for lo, hi in [(0.0, 1000.0), (100.0, 100.1), (-73.25, -20.0), (-1.0, 1.0)]:
        st, c, s = oracle.map_constants(lo, hi, True)
        assert st == "ok"
        assert c == float(np.float32(c)) and s == float(np.float32(s))
        assert abs(c - (lo + hi) / 2) <= 1e-7 * max(abs(lo), abs(hi))
        assert abs(s * (hi - lo) / 2 - 1.0) <= 1e-7
        # rounding c to FP32 shifts the mapped interval by at most s * |c| * 2^-24
        t = s * (np.array([lo, hi]) - c)
        assert np.all(np.abs(np.abs(t) - 1.0) <= s * abs(c) * 2.0 ** -24 + 1e-6)
        st, c64, s64 = oracle.map_constants(lo, hi, False)
        assert c64 == (lo + hi) / 2 and s64 == 2.0 / (hi - lo)


def _compose_exact(Xt, c, s):
    """x-basis coefficients of sum_k Xt[k] (s x - s c)^k by repeated polynomial products."""
    c = Fraction(c)
    s = Fraction(s)
    out = [Fraction(0)] * len(Xt)
    power = [Fraction(1)]  # (s x - s c)^k, ascending
    for k, a in enumerate(Xt):
        for j, p in enumerate(power):
            out[j] += Fraction(a) * p
        nxt = [Fraction(0)] * (len(power) + 1)
        for j, p in enumerate(power):
            nxt[j] += -s * c * p
            nxt[j + 1] += s * p
        power = nxt
    return out


@pytest.mark.parametrize("m", [1, 3, 5, 8])
def test_unmap_against_exact_composition(m):
    rng = np.random.default_rng(1000 + m)
    Xt = rng.normal(size=m + 1)
    _, c, s = oracle.map_constants(-3.0, 11.0, True)
    X = oracle.unmap(Xt, c, s)
    ref = [float(v) for v in _compose_exact(list(Xt), c, s)]
    scale = [sum(abs(float(v)) for v in _compose_exact(list(np.abs(Xt)), -abs(c), s))] * (m + 1)
    np.testing.assert_array_less(np.abs(X - ref), 1e-13 * np.array(scale) + 1e-300)


def test_mapped_fit_equals_direct_fit():
    d = synth.single_fp64(20000, seed=11)
    for m in (1, 2, 3):
        direct = oracle.fit(d["x"], d["y"], m)
        mapped = oracle.fit_interval(d["x"], d["y"], m, 0.0, 10.0, fp32=False)
        assert mapped["status"] == "ok"
        np.testing.assert_allclose(mapped["X"], direct["X"], rtol=1e-8, atol=1e-9)
        # the mapped sums are those of t = s (x - c)
        t = mapped["s"] * (d["x"] - mapped["c"])
        assert abs(mapped["S"][1] - np.sum(t)) <= 1e-9 * np.sum(np.abs(t))


# --- statistics of the FP64 single-series workload ----------------------------------------

def test_single_fp64_statistics():
    d = synth.single_fp64()
    out = oracle.fit(d["x"], d["y"], 3)
    assert out["status"] == "ok"
    Ainv = np.linalg.inv(_hankel(out["S"], 3))
    sd = d["sigma"] * np.sqrt(np.diag(Ainv))
    assert np.all(np.abs(out["X"] - d["true"]) <= 5 * sd), (out["X"], d["true"], sd)


# --- the adjoint: finite differences and autograd -------------------------------------------

def _loss(x, y, m, cs, w):
    out = oracle.fit(x, y, m, cs)
    return float(np.sum(w * out["X"] ** 2))


@pytest.mark.parametrize("mapped", [False, True])
def test_backward_central_differences(mapped):
    rng = np.random.default_rng(1200 + int(mapped))
    m = 3
    n = 64
    if mapped:
        x = rng.uniform(2.0, 6.0, n)
        st, c, s = oracle.map_constants(2.0, 6.0, True)
        cs = (c, s)
    else:
        x = rng.uniform(-1.0, 1.0, n)
        cs = None
    y = 0.5 + x - 0.3 * x ** 2 + rng.normal(0.0, 0.05, n)
    w = rng.normal(size=m + 1)
    out = oracle.fit(x, y, m, cs)
    gX = 2.0 * w * out["X"]
    st, dx, dy = oracle.backward(x, y, m, cs, out["S"], out["Xt"], gX)
    assert st == "ok"
    h = 1e-6
    for i in range(0, n, 5):
        yp, ym = y.copy(), y.copy()
        yp[i] += h
        ym[i] -= h
        fd_y = (_loss(x, yp, m, cs, w) - _loss(x, ym, m, cs, w)) / (2 * h)
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd_x = (_loss(xp, y, m, cs, w) - _loss(xm, y, m, cs, w)) / (2 * h)
        assert abs(fd_y - dy[i]) <= 1e-6 * (np.max(np.abs(dy)) + 1e-12)
        assert abs(fd_x - dx[i]) <= 1e-6 * (np.max(np.abs(dx)) + 1e-12)


def test_backward_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1300)
    m, n = 3, 500
    lo, hi = -2.0, 5.0
    x = rng.uniform(lo, hi, n)
    y = np.sin(x) + rng.normal(0.0, 0.1, n)
    w = rng.normal(size=m + 1)
    _, c, s = oracle.map_constants(lo, hi, True)
    out = oracle.fit(x, y, m, (c, s))
    st, dx, dy = oracle.backward(x, y, m, (c, s), out["S"], out["Xt"], 2.0 * w * out["X"])
    assert st == "ok"
    # restatement in torch FP64 with library linear algebra; autograd differentiates it
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    yt = torch.tensor(y, dtype=torch.float64, requires_grad=True)
    t = s * (xt - c)
    P = torch.stack([t ** k for k in range(2 * m + 1)], dim=1)
    Ssum = P.sum(0)
    Tsum = (P[:, : m + 1] * yt[:, None]).sum(0)
    A = torch.stack([Ssum[j: j + m + 1] for j in range(m + 1)])
    Xt = torch.linalg.solve(A, Tsum)
    M = torch.zeros(m + 1, m + 1, dtype=torch.float64)
    from math import comb
    for j in range(m + 1):
        for k in range(j, m + 1):
            M[j, k] = comb(k, j) * s ** k * (-c) ** (k - j)
    X = M @ Xt
    L = (torch.tensor(w) * X ** 2).sum()
    L.backward()
    np.testing.assert_allclose(X.detach().numpy(), out["X"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(dy, yt.grad.numpy(), rtol=1e-7, atol=1e-9 * np.max(np.abs(dy)))
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-7, atol=1e-9 * np.max(np.abs(dx)))


# --- the alternative solver: Cholesky of the SPD Hankel matrix (Section V) -----------------

@pytest.mark.parametrize("m", [1, 2, 3, 5, 8])
def test_cholesky_against_lapack_and_gauss(m):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    d = synth.small_series(3000, seed=1400 + m, m=m, noise=0.05, dtype=np.float64)
    S, T = oracle.powersums(d["x"], d["y"], m)
    st, X = oracle.solve_cholesky(S, T, m)
    assert st == "ok"
    A = _hankel(S, m)
    ref = scipy_linalg.cho_solve(scipy_linalg.cho_factor(A, lower=True), T)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 1e2 * cond * EPS
    st2, Xg = oracle.solve(S, T, m)
    assert np.linalg.norm(X - Xg) / np.linalg.norm(Xg) <= 1e2 * cond * EPS


def test_cholesky_table1_and_statuses():
    _, _, x, y = _table1()
    for m in (1, 2, 3):
        S, T = oracle.powersums(x, y, m)
        st, X = oracle.solve_cholesky(S, T, m)
        assert st == "ok"
        np.testing.assert_allclose(X, oracle.fit(x, y, m)["X"], rtol=1e-6)
    S, T = oracle.powersums(np.full(10, 2.0), np.arange(10.0), 1)
    assert oracle.solve_cholesky(S, T, 1)[0] == "singular"
    S, T = oracle.powersums(np.array([1.0, 2.0, 3.0]), np.array([1.0, np.nan, 3.0]), 1)
    assert oracle.solve_cholesky(S, T, 1)[0] == "nonfinite"


# --- Generalised objective: per-point weights and the Chebyshev basis ----------------

def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.mark.parametrize("m", [1, 3, 5])
def test_weighted_against_lstsq(m):
    """Weighted LSE = ordinary least squares of the sqrt(w)-scaled Vandermonde system."""
    rng = np.random.default_rng(1500 + m)
    x = rng.uniform(-1.0, 1.0, 800)
    y = np.polynomial.polynomial.polyval(x, rng.normal(size=m + 1)) + rng.normal(0, 0.05, x.size)
    w = rng.uniform(0.05, 3.0, x.size)
    r = oracle.fit_general(x, y, m, w=w)
    assert r["status"] == "ok"
    V = np.vander(x, m + 1, increasing=True) * np.sqrt(w)[:, None]
    ref = np.linalg.lstsq(V, y * np.sqrt(w), rcond=None)[0]
    cond = np.linalg.cond(r["G"])
    assert _rel(r["X"], ref) <= 1e2 * cond * EPS
    # the weights matter: the unweighted fit differs
    assert _rel(oracle.fit(x, y, m)["X"], ref) > 1e3 * cond * EPS


@pytest.mark.parametrize("basis", ["monomial", "chebyshev"])
def test_integer_weights_are_repeated_points(basis):
    """An integer weight w_i is the point (x_i, y_i) taken w_i times (brute force)."""
    rng = np.random.default_rng(1510)
    x = rng.uniform(-2.0, 3.0, 60)
    y = rng.normal(size=x.size)
    w = rng.integers(0, 5, x.size).astype(np.float64)
    m = 3
    cs = (0.5, 0.4)
    r = oracle.fit_general(x, y, m, w=w, basis=basis, cs=cs)
    xr, yr = np.repeat(x, w.astype(int)), np.repeat(y, w.astype(int))
    ref = oracle.fit_interval(xr, yr, m, -2.0, 3.0, fp32=False)
    assert r["status"] == "ok" and ref["status"] == "ok"
    cond = np.linalg.cond(r["G"])
    assert _rel(r["X"], ref["X"]) <= 1e3 * cond * EPS


@pytest.mark.parametrize("m", [2, 4, 8, 12, 16])
def test_chebyshev_against_chebfit(m):
    """Chebyshev coefficients of the (weighted) fit equal numpy's chebfit, an
    independent least-squares solve of the Chebyshev-Vandermonde system."""
    rng = np.random.default_rng(1520 + m)
    t = rng.uniform(-1.0, 1.0, 1500)
    y = np.cos(3 * t) + rng.normal(0, 0.01, t.size)
    w = rng.uniform(0.2, 2.0, t.size)
    for ww in (None, w):
        r = oracle.fit_general(t, y, m, w=ww, basis="chebyshev")
        assert r["status"] == "ok"
        ref = np.polynomial.chebyshev.chebfit(t, y, m, w=None if ww is None else np.sqrt(ww))
        assert _rel(r["Xb"], ref) <= 1e3 * np.linalg.cond(r["G"]) * EPS


def test_chebyshev_nodes_closed_form():
    """At the n Chebyshev nodes t_i = cos(pi (i + 1/2) / n) the basis is
    discretely orthogonal: G = diag(n, n/2, ..., n/2) and a_k = (2/n) sum_i
    y_i cos(k theta_i) (a_0 with 1/n)."""
    n, m = 64, 7
    theta = np.pi * (np.arange(n) + 0.5) / n
    t = np.cos(theta)
    y = np.exp(t) * np.sin(2 * t)
    r = oracle.fit_general(t, y, m, basis="chebyshev")
    assert r["status"] == "ok"
    np.testing.assert_allclose(r["G"], np.diag([n] + [n / 2] * m), atol=1e-12 * n)
    a = np.array([(1.0 if k == 0 else 2.0) / n * np.sum(y * np.cos(k * theta)) for k in range(m + 1)])
    np.testing.assert_allclose(r["Xb"], a, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("m", [1, 3, 6, 9])
def test_cheb_to_mono_against_numpy(m):
    a = np.random.default_rng(1530 + m).normal(size=m + 1)
    np.testing.assert_allclose(oracle.cheb_to_mono(a), np.polynomial.chebyshev.cheb2poly(a),
                               rtol=1e-13, atol=1e-13 * 2.0 ** m)


def test_chebyshev_and_monomial_fit_the_same_polynomial():
    """Both bases span the polynomials of degree <= m, so the minimiser is the
    same function: equal x-basis coefficients (Table I, mapped and not)."""
    _, _, x, y = _table1()
    for m in (1, 2, 3):
        ref = oracle.fit(x, y, m)["X"]
        for cs in (None, (np.mean(x), 2.0 / (x.max() - x.min()))):
            r = oracle.fit_general(x, y, m, basis="chebyshev", cs=cs)
            assert r["status"] == "ok"
            assert _rel(r["X"], ref) <= 1e-8
        rw = oracle.fit_general(x, y, m, w=np.ones_like(x))
        assert _rel(rw["X"], ref) <= 1e-8


def test_general_statuses():
    x = np.array([0.0, 1.0, 2.0])
    assert oracle.fit_general(x, x, 3, basis="chebyshev")["status"] == "n_too_small"
    assert oracle.fit_general(x, x, 2, w=np.array([1.0, 0.0, 1.0]))["status"] == "singular"
    assert oracle.fit_general(x, np.array([0.0, np.nan, 1.0]), 1, basis="chebyshev")["status"] == "nonfinite"
    assert oracle.fit_general(x, x, 1, w=np.array([1.0, np.inf, 1.0]))["status"] == "nonfinite"
    assert oracle.fit_general(np.full(5, 0.3), np.arange(5.0), 1, basis="chebyshev")["status"] == "singular"
    assert oracle.fit_general_interval(x, x, 1, 1.0, 1.0, fp32=False)["status"] == "bad_interval"


# --- residuals in either basis (Section III, Table V) -----------------------------------

@pytest.mark.parametrize("basis", ["monomial", "chebyshev"])
def test_residuals_general_against_numpy(basis):
    """r, SSE and V^T r of an arbitrary polynomial against numpy's own evaluation
    (polyval / chebval) and Vandermonde matrices (vander / chebvander)."""
    rng = np.random.default_rng(1540)
    x = rng.uniform(2.0, 9.0, 777)
    y = rng.normal(size=x.size)
    Xb = rng.normal(size=6)
    c, s = 5.5, 2.0 / 7.0
    t = s * (x - c)
    if basis == "chebyshev":
        f = np.polynomial.chebyshev.chebval(t, Xb)
        V = np.polynomial.chebyshev.chebvander(t, 5)
    else:
        f = np.polynomial.polynomial.polyval(t, Xb)
        V = np.vander(t, 6, increasing=True)
    sse, vtr, r = oracle.residuals_general(x, y, Xb, basis, cs=(c, s))
    np.testing.assert_allclose(r, y - f, rtol=0, atol=1e-13)
    assert abs(sse - np.sum((y - f) ** 2)) <= 1e-12 * sse
    np.testing.assert_allclose(vtr, V.T @ (y - f), rtol=0, atol=1e-11)


def test_residuals_general_table1_and_orthogonality():
    """Table I, m = 3: the SSE of the exact fit (128.1995754) in both bases, with
    V^T r = 0 at the least-squares solution (the normal equations of Section II)."""
    _, _, x, y = _table1()
    cs = (np.mean(x), 2.0 / (x.max() - x.min()))
    mono = oracle.fit(x, y, 3)
    sse_m, vtr_m, _ = oracle.residuals_general(x, y, mono["X"], "monomial")
    assert abs(sse_m - oracle.sse(mono["X"], x, y)) <= 1e-12 * sse_m
    assert abs(sse_m - 128.1995754) <= 1e-6
    cheb = oracle.fit_general(x, y, 3, basis="chebyshev", cs=cs)
    sse_c, vtr_c, _ = oracle.residuals_general(x, y, cheb["Xb"], "chebyshev", cs=cs)
    assert abs(sse_c - sse_m) <= 1e-9 * sse_m
    scale = np.sum(np.abs(y)) * 1e3
    assert np.max(np.abs(vtr_c)) <= 1e-12 * scale
    assert np.max(np.abs(vtr_m[:1])) <= 1e-9 * scale


# --- the all-core timing variant of the power sums -----------------------------------------

@pytest.mark.parametrize("threads", [1, 2, 3, 8, 16])
@pytest.mark.parametrize("m", [1, 3, 8])
def test_powersums_threads_bit_exact_int(threads, m):
    """Small integers: every partial sum is an exact FP64 integer, so any order of
    addition gives the exact power sums: the all-core variant equals int64 sums."""
    rng = np.random.default_rng(900 + threads + m)
    n = 10_007
    xi = rng.integers(-6, 7, n)
    yi = rng.integers(-50, 51, n)
    S, T = oracle.powersums_threads(xi.astype(np.float64), yi.astype(np.float64), m, threads=threads)
    x64 = xi.astype(np.int64)
    assert S[0] == n
    for k in range(1, 2 * m + 1):
        assert S[k] == float(int(np.sum(x64 ** k))), k
    for k in range(m + 1):
        assert T[k] == float(int(np.sum(x64 ** k * yi))), k


@pytest.mark.parametrize("threads", [2, 5, 16])
def test_powersums_threads_within_the_summation_bound(threads):
    """Random data: the all-core sums and the sequential oracle's add the same
    terms in different orders, so they differ by at most twice the bound of one
    recursive sum, 2 (n - 1) 2^-53 sum |t|^k (|y|), and are repeatable."""
    d = synth.single_large(n=200_003, m=3, seed=901)
    x, y = d["x"].astype(np.float64), d["y"].astype(np.float64)
    cs = (0.25, 1.5)
    for m in (1, 4):
        S1, T1 = oracle.powersums(x, y, m, cs)
        St, Tt = oracle.powersums_threads(x, y, m, cs, threads=threads)
        t = cs[1] * (x - cs[0])
        Sa, Ta = oracle.powersums(np.abs(t), np.abs(y), m)
        bound = 2 * (x.size - 1) * 2.0 ** -53
        assert St[0] == S1[0] == x.size
        assert np.all(np.abs(St[1:] - S1[1:]) <= bound * Sa[1:])
        assert np.all(np.abs(Tt - T1) <= bound * Ta)
        S2, T2 = oracle.powersums_threads(x, y, m, cs, threads=threads)
        assert np.array_equal(St, S2) and np.array_equal(Tt, T2)
    # one thread is the sequential routine itself
    S1, T1 = oracle.powersums(x, y, 2)
    S2, T2 = oracle.powersums_threads(x, y, 2, threads=1)
    assert np.array_equal(S1, S2) and np.array_equal(T1, T2)


def test_powersums_threads_edges():
    # fewer points than threads (empty ranges), no points, bad thread counts
    S, T = oracle.powersums_threads(np.array([1.0, 2.0, 3.0]), np.array([1.0, 1.0, 1.0]), 2, threads=8)
    assert list(S) == [3.0, 6.0, 14.0, 36.0, 98.0] and list(T) == [3.0, 6.0, 14.0]
    S, T = oracle.powersums_threads(np.zeros(0), np.zeros(0), 1, threads=4)
    assert list(S) == [0.0, 0.0, 0.0] and list(T) == [0.0, 0.0]
    for bad in (0, -1, 5000):
        with pytest.raises(ValueError):
            oracle.powersums_threads(np.ones(4), np.ones(4), 1, threads=bad)


def test_fit_threads_matches_fit():
    d = synth.single_fp64(n=50_000)
    a = oracle.fit(d["x"], d["y"], 3)
    b = oracle.fit_threads(d["x"], d["y"], 3, threads=6)
    assert a["status"] == b["status"] == "ok"
    assert np.linalg.norm(a["X"] - b["X"]) <= 1e-9 * np.linalg.norm(a["X"])
    st, c, s = oracle.map_constants(0.0, 10.0, False)
    a = oracle.fit(d["x"], d["y"], 2, (c, s))
    b = oracle.fit_threads(d["x"], d["y"], 2, (c, s), threads=3)
    assert np.linalg.norm(a["X"] - b["X"]) <= 1e-12 * np.linalg.norm(a["X"])
    assert np.linalg.norm(a["Xt"] - b["Xt"]) <= 1e-12 * np.linalg.norm(a["Xt"])
