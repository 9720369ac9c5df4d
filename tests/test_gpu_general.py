"""Parity of the generalised single-series fit (lsefit_fit_general: per-point
weights, Chebyshev basis) with the oracle's fit_general.

The oracle fits the stored (dequantised) values in FP64 from the definition
G[j][k] = sum w phi_j phi_k; the kernels accumulate the 2m+1 moments and use
the product identity of the Chebyshev polynomials.  Tolerances (relative
2-norm error of the basis coefficients Xb, policy of tests/gates.py):
max(1e-6, cond(G) 2^-53 4m) for FP64 accumulation; max(1e-5, cond(G) 2^-24 4m)
for compensated FP32 (the per-point basis values carry about k 2^-24 relative
error); naive FP32 adds the summation error, floored here at 1e-4 for the
sizes used.  Gates above 1e-3 are not applied (reported); the backward error
of Xb in the oracle's normal equations G Xb = b is gated always.  Statuses
must match the oracle's.
"""
import numpy as np
import pytest

import gates
import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def L():
    import paper_1512_08017_gb300 as lib
    return lib


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _base(accum):
    return 1e-4 if accum == "naive" else None


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _stored(t):
    return t.double().cpu().numpy()


def _check(L, out, ref, accum, m, row=0, n=1 << 24):
    st = L.status_names(out["status"])[row]
    assert st == ref["status"], (st, ref["status"])
    if st != "ok":
        assert np.all(np.isnan(out["X"][row, : m + 1].cpu().numpy()))
        return None
    e, _, _ = gates.check_coefficients(out["Xb"][row, : m + 1].cpu().numpy(), ref["Xb"], ref["G"], ref["b"],
                                       accum, m, _base(accum), n=n)
    return e


@pytest.mark.parametrize("accum", ["comp", "naive", "f64"])
@pytest.mark.parametrize("m", [1, 3, 5])
def test_weighted_unit_interval(L, accum, m):
    n = (1 << 20) + 13
    d = synth.single_large(n=n, m=m, seed=60 + m)
    w = synth.weights(n, seed=61 + m)
    x, y, wd = _dev(d["x"]), _dev(d["y"]), _dev(w)
    fp32 = accum != "f64"
    ref = oracle.fit_general_interval(_stored(x), _stored(y), m, -1.0, 1.0, fp32=fp32, w=_stored(wd))
    out = L.fit_general(x, y, m, w=wd, accum=accum, interval=(-1.0, 1.0))
    _check(L, out, ref, accum, m)
    # the mapped constants are the oracle's
    mp = out["map"].cpu().numpy()
    assert mp[0] == ref["c"] and mp[1] == ref["s"]


@pytest.mark.parametrize("accum", ["comp", "f64"])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
def test_chebyshev_unscaled_interval(L, accum, m):
    """x on [0, 1000] mapped to [-1, 1]: the Chebyshev normal matrix stays well
    conditioned at every degree (the monomial Hankel matrix reaches ~1e6 at
    m = 8), so the FP32 bound stays near 1e-5 at every degree."""
    d = synth.precision(n=1 << 20, m=m)
    lo, hi = d["interval"]
    x, y = _dev(d["x"]), _dev(d["y"])
    fp32 = accum != "f64"
    ref = oracle.fit_general_interval(_stored(x), _stored(y), m, lo, hi, fp32=fp32, basis="chebyshev")
    assert np.linalg.cond(ref["G"]) < 100.0
    out = L.fit_general(x, y, m, basis="chebyshev", accum=accum, interval=(lo, hi))
    _check(L, out, ref, accum, m)


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("m", [4, 8])
def test_full_grid_iterations(L, m, weighted, offset):
    """Enough points for several full iterations of the FP32 pass's main loop
    at the largest grid, plus a ragged tail.  At degree 8 one iteration takes
    152 blocks x 256 threads x 8 vectors (about 1.25M points), so smaller
    cases run only the tail loop.  Degree 8 runs the register pipeline with the
    per-thread L2 prefetch (unweighted) or the prefetch alone (weighted); degree 4
    runs the block prefetch.  offset 1 starts x, y (and w) one element past a
    16-byte boundary (three scalar head points)."""
    n = 3 * 1_245_184 + 4097
    d = synth.precision(n=n + offset, m=m, seed=97)
    lo, hi = d["interval"]
    x = _dev(d["x"])[offset:]
    y = _dev(d["y"])[offset:]
    wd = _dev(synth.weights(n + offset, seed=98))[offset:] if weighted else None
    ref = oracle.fit_general_interval(_stored(x), _stored(y), m, lo, hi, fp32=True,
                                      w=_stored(wd) if weighted else None, basis="chebyshev")
    out = L.fit_general(x, y, m, w=wd, basis="chebyshev", accum="comp", interval=(lo, hi))
    _check(L, out, ref, "comp", m, n=n)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("m", [6, 7, 8])
def test_unweighted_monomial_high_degree(L, m, dtype):
    """The unweighted pass above degree 5 in the monomial basis (its slots are
    split over warp pairs), compensated and naive, against the oracle."""
    n = 2 * 1_245_184 + 777
    d = synth.small_series(n, seed=99 + m, lo=-2.0, hi=6.0, m=m, dtype=np.float64)
    x, y = _dev(d["x"], dtype), _dev(d["y"], dtype)
    for accum in ("comp", "naive"):
        ref = oracle.fit_general_interval(_stored(x), _stored(y), m, -2.0, 6.0, fp32=True)
        out = L.fit_general(x, y, m, accum=accum, interval=(-2.0, 6.0))
        _check(L, out, ref, accum, m, n=n)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
@pytest.mark.parametrize("m", [2, 5, 6, 8])
def test_weighted_chebyshev_storage(L, dtype, m):
    n = 300_001
    d = synth.small_series(n, seed=70 + m, lo=-3.0, hi=5.0, m=m, dtype=np.float64)
    w = synth.weights(n, seed=71 + m)
    x, y, wd = _dev(d["x"], dtype), _dev(d["y"], dtype), _dev(w, dtype)
    accums = ["f64"] if dtype == torch.float64 else ["comp", "f64"]
    for accum in accums:
        fp32 = accum != "f64"
        ref = oracle.fit_general_interval(_stored(x), _stored(y), m, -3.0, 5.0, fp32=fp32, w=_stored(wd),
                                          basis="chebyshev")
        out = L.fit_general(x, y, m, w=wd, basis="chebyshev", accum=accum, interval=(-3.0, 5.0))
        _check(L, out, ref, accum, m)


@pytest.mark.parametrize("basis", ["monomial", "chebyshev"])
@pytest.mark.parametrize("weighted", [False, True])
def test_nested_degrees(L, basis, weighted):
    if basis == "monomial" and not weighted:
        pytest.skip("the paper's objective: covered by the lsefit_fit tests")
    n, m, m_lo = 200_003, 6, 2
    d = synth.small_series(n, seed=80, m=m)
    w = synth.weights(n, seed=81) if weighted else None
    x, y = _dev(d["x"]), _dev(d["y"])
    wd = _dev(w) if weighted else None
    out = L.fit_general(x, y, m, w=wd, basis=basis, m_lo=m_lo, accum="comp", interval=(-1.0, 1.0))
    for row, deg in enumerate(range(m_lo, m + 1)):
        ref = oracle.fit_general_interval(_stored(x), _stored(y), deg, -1.0, 1.0, fp32=True,
                                          w=_stored(wd) if weighted else None, basis=basis)
        _check(L, out, ref, "comp", deg, row)
        assert np.all(out["X"][row, deg + 1:].cpu().numpy() == 0.0)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 9, 33, 1000, 4097, 65537])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
def test_sums_sizes_and_alignment(L, n, dtype):
    """Moments and right-hand sides against a Chebyshev-Vandermonde product
    (numpy, FP64) for ragged sizes and every alignment of x, y, w."""
    m = 3
    d = synth.small_series(n + 3, seed=90 + n, m=m, dtype=np.float64)
    wv = synth.weights(n + 3, seed=91 + n).astype(np.float64)
    xs, ys, ws = (torch.from_numpy(a).to(dtype) for a in (d["x"], d["y"], wv))
    accum = "f64" if dtype == torch.float64 else "comp"
    for ox, oy, ow in [(0, 0, 0), (1, 1, 1), (1, 2, 1), (3, 3, 2)]:
        x = xs.cuda()[ox: ox + n]
        y = ys.cuda()[oy: oy + n]
        w = ws.cuda()[ow: ow + n]
        out = L.fit_general(x, y, m, w=w, basis="chebyshev", accum=accum)
        xr, yr, wr = _stored(x), _stored(y), _stored(w)
        V = np.polynomial.chebyshev.chebvander(xr, 2 * m)
        mom = (wr[:, None] * V).sum(axis=0)
        rhs = (wr[:, None] * V[:, : m + 1] * yr[:, None]).sum(axis=0)
        # |T_p(t)| <= 1 on [-1, 1]; the recurrence's rounding error grows like p^2 eps
        p2 = np.arange(2 * m + 1) ** 2 + 1.0
        scale_m = np.abs(wr).sum() * p2
        scale_r = np.abs(wr * yr).sum() * p2[: m + 1]
        got = out["sums"].cpu().numpy()
        tol = 1e-13 if accum == "f64" else 8 * EPS32
        assert np.all(np.abs(got[: 2 * m + 1] - mom) <= tol * scale_m + 1e-300), (ox, oy, ow)
        assert np.all(np.abs(got[2 * m + 1:] - rhs) <= tol * scale_r + 1e-300), (ox, oy, ow)
        st = L.status_names(out["status"])[0]
        assert st == ("n_too_small" if n < m + 1 else "ok")


def test_statuses(L):
    f32 = torch.float32
    x = _dev(np.linspace(-1, 1, 1000), f32)
    y = _dev(np.cos(np.linspace(-1, 1, 1000)), f32)
    ones = torch.ones_like(x)
    # zero weights everywhere: singular
    out = L.fit_general(x, y, 2, w=torch.zeros_like(x), basis="chebyshev")
    assert L.status_names(out["status"]) == ["singular"]
    # NaN weight: nonfinite
    wn = ones.clone()
    wn[17] = float("nan")
    assert L.status_names(L.fit_general(x, y, 2, w=wn)["status"]) == ["nonfinite"]
    # all-equal abscissae: singular
    assert L.status_names(L.fit_general(torch.full_like(x, 0.25), y, 1, basis="chebyshev")["status"]) == ["singular"]
    # too few points, bad interval
    assert L.status_names(L.fit_general(x[:3], y[:3], 3, w=ones[:3])["status"]) == ["n_too_small"]
    assert L.status_names(L.fit_general(x, y, 2, w=ones, interval=(1.0, 1.0))["status"]) == ["bad_interval"]
    # unit weights: the unweighted fit
    a = L.fit_general(x, y, 3, w=ones, accum="f64")["X"].cpu().numpy()
    b = L.fit(x, y, 3, accum="f64")["X"].cpu().numpy()
    assert _rel(a, b) <= 1e-9


def test_integer_weights_are_repeated_points(L):
    """A point of integer weight k counts as k copies (GPU against GPU: the
    general pass with weights against lsefit_fit on repeated points)."""
    rng = np.random.default_rng(95)
    n = 50_000
    x = rng.uniform(-1, 1, n).astype(np.float32)
    y = (np.sin(3 * x) + rng.normal(0, 0.01, n)).astype(np.float32)
    k = rng.integers(0, 4, n)
    out = L.fit_general(_dev(x), _dev(y), 4, w=_dev(k.astype(np.float32)), accum="f64")
    rep = L.fit(_dev(np.repeat(x, k)), _dev(np.repeat(y, k)), 4, accum="f64")
    assert _rel(out["X"].cpu().numpy(), rep["X"].cpu().numpy()) <= 1e-9


def test_monomial_without_weights_is_lsefit_fit(L):
    d = synth.small_series(100_000, seed=96, m=3)
    x, y = _dev(d["x"]), _dev(d["y"])
    a = L.fit_general(x, y, 3, m_lo=1)
    b = L.fit_degrees(x, y, 3, m_lo=1)
    assert torch.equal(a["X"], b["X"]) and torch.equal(a["Xb"], b["Xt"])


def test_invalid_arguments(L):
    x = _dev(np.zeros(10))
    with pytest.raises(ValueError):
        L.fit_general(x, x, 2, basis="legendre")
    with pytest.raises(ValueError):
        L.fit_general(x, x, 9)
    with pytest.raises(ValueError):
        L.fit_general(x, x, 2, w=_dev(np.zeros(9)))
    from paper_1512_08017_gb300 import lsefit as B
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    X = torch.empty(3, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = B.lib.lsefit_fit_general(B._ptr(x), B._ptr(x), None, 10, B.F64, 2, 2, 1, 1, None, B._ptr(X), None,
                                  None, None, B._ptr(st), B._ptr(ws), ws.numel(), None)
    assert rc == B.ERR_UNSUPPORTED  # F64 storage needs F64 accumulation
    rc = B.lib.lsefit_fit_general(B._ptr(x), B._ptr(x), None, 10, B.F64, 2, 2, 2, 5, None, B._ptr(X), None,
                                  None, None, B._ptr(st), B._ptr(ws), ws.numel(), None)
    assert rc == B.ERR_INVALID_ARG
    rc = B.lib.lsefit_fit_general(B._ptr(x), B._ptr(x), None, 10, B.F64, 2, 2, 2, 1, None, B._ptr(X), None,
                                  None, None, B._ptr(st), B._ptr(ws), 1024, None)
    assert rc == B.ERR_WORKSPACE


def test_full_size_weighted(L):
    """The weighted workload at its benchmark size (2^28 FP32 points on
    [-1, 1], m = 3, compensated): whole-series parity with the oracle."""
    n = 1 << 28
    d = synth.single_large(n=n, m=3)
    w = synth.weights(n)
    x, y, wd = _dev(d["x"]), _dev(d["y"]), _dev(w)
    out = L.fit_general(x, y, 3, w=wd, accum="comp", interval=(-1.0, 1.0))
    del x, y, wd
    ref = oracle.fit_general_interval(d["x"], d["y"], 3, -1.0, 1.0, fp32=True, w=w)
    _check(L, out, ref, "comp", 3)


def test_mapped_host_memory(L):
    """Points and weights in pinned host memory are streamed by the kernel directly."""
    n = (1 << 18) + 7
    d = synth.small_series(n, seed=97, m=3)
    w = synth.weights(n, seed=98)
    x, y, wh = (torch.from_numpy(a).pin_memory() for a in (d["x"], d["y"], w))
    out = L.fit_general(x, y, 3, w=wh, basis="chebyshev", accum="comp", interval=(-1.0, 1.0))
    ref = oracle.fit_general_interval(d["x"].astype(np.float64), d["y"].astype(np.float64), 3, -1.0, 1.0,
                                      fp32=True, w=w.astype(np.float64), basis="chebyshev")
    _check(L, out, ref, "comp", 3)


@pytest.mark.parametrize("m", [9, 12, 16])
@pytest.mark.parametrize("weighted", [False, True])
def test_chebyshev_high_degrees(L, m, weighted):
    """Degrees above 8 in the Chebyshev basis with FP64 accumulation (x on
    [0, 1000] mapped): the normal matrix stays well conditioned where the
    monomial one is singular at the FP64 threshold."""
    d = synth.precision(n=1 << 20, m=m)
    lo, hi = d["interval"]
    w = synth.weights(1 << 20, seed=99) if weighted else None
    x, y = _dev(d["x"]), _dev(d["y"])
    wd = _dev(w) if weighted else None
    xs, ys = _stored(x), _stored(y)
    ref = oracle.fit_general_interval(xs, ys, m, lo, hi, fp32=False, w=_stored(wd) if weighted else None,
                                      basis="chebyshev")
    assert np.linalg.cond(ref["G"]) < 1e3
    out = L.fit_general(x, y, m, w=wd, basis="chebyshev", m_lo=m - 2, accum="f64", interval=(lo, hi))
    _check(L, out, ref, "f64", m, row=2)
    # the same degree in the monomial basis: a normal matrix orders of magnitude worse
    # conditioned (singular at the FP64 threshold from about m = 12)
    mono = oracle.fit_general_interval(xs, ys, m, lo, hi, fp32=False, basis="monomial")
    assert mono["status"] == "singular" or np.linalg.cond(mono["G"]) > 1e3 * np.linalg.cond(ref["G"])


def test_chebyshev_high_degree_limits(L):
    x = _dev(np.linspace(-1, 1, 1000))
    with pytest.raises(L.LsefitError):  # FP32 accumulation is limited to degree 8
        L.fit_general(x, x, 9, basis="chebyshev", accum="comp")
    with pytest.raises(ValueError):
        L.fit_general(x, x, 9, basis="monomial", accum="f64")
    with pytest.raises(ValueError):
        L.fit_general(x, x, 17, basis="chebyshev", accum="f64")

