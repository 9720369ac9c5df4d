"""Parity of the residual pass (lsefit_residuals) with the oracle.

SSE and V^T r are compared with the oracle's residuals of its own fit of the
same stored points, evaluated in the mapped basis in FP64.  Tolerance: SSE
relative 1e-4 for FP32 data (the residual r = y - f(t) is formed in FP32 and
loses up to |y|/|r| of its 2^-24 relative precision), 1e-9 for FP64 data;
V^T r absolute, scaled by sum_i |t_i^k| |y_i| times the same factor.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import read_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_1512_08017_gb300 as lib
    return lib


def _ref(xs, ys, m, lo, hi, fp32):
    r = oracle.fit_interval(xs, ys, m, lo, hi, fp32=fp32)
    t = r["s"] * (xs - r["c"])
    res = ys - oracle.evaluate(r["Xt"], t)
    vtr = np.array([np.sum(t ** k * res) for k in range(m + 1)])
    scale = np.array([np.sum(np.abs(t) ** k * np.abs(ys)) for k in range(m + 1)])
    return r, float(np.sum(res * res)), vtr, scale, res


@pytest.mark.parametrize("dtype,accum", [(torch.float32, "comp"), (torch.float64, "f64"),
                                         (torch.bfloat16, "comp")])
@pytest.mark.parametrize("tuning", [None, {"warp_max_len": 256, "chunk_len": 4096}])
def test_residuals_against_oracle(L, dtype, accum, tuning):
    b = synth.ragged_batch(num_series=150, lmin=20, lmax=30000, seed=91)
    x = torch.from_numpy(b["x"]).to(dtype).cuda()
    y = torch.from_numpy(b["y"]).to(dtype).cuda()
    xs = x.double().cpu().numpy()  # the stored values
    ys = y.double().cpu().numpy()
    plan = L.BatchPlan(b["offsets"], 5, tuning=tuning, degree=b["degree"])
    fwd = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, accum=accum, plan=plan)
    out = L.residuals_batched(x, y, b["offsets"], b["degree"], fwd, want_r=True)
    sse = out["sse"].cpu().numpy()
    vtr = out["vtr"].cpu().numpy()
    rr = out["r"].double().cpu().numpy()
    tol = 1e-9 if dtype == torch.float64 else (1e-4 if dtype == torch.float32 else 1e-3)
    checked = 0
    for s in range(150):
        lo, hi = int(b["offsets"][s]), int(b["offsets"][s + 1])
        m = int(b["degree"][s])
        if L.status_names(fwd["status"][s: s + 1]) != ["ok"]:
            continue
        r, sse_ref, vtr_ref, scale, res = _ref(xs[lo:hi], ys[lo:hi], m, *b["interval"][s], fp32=accum != "f64")
        assert abs(sse[s] - sse_ref) <= tol * sse_ref + 1e-30, (s, sse[s], sse_ref)
        f = 8 * m * (2.0 ** -53 if accum == "f64" else 2.0 ** -24)
        assert np.all(np.abs(vtr[s, : m + 1] - vtr_ref) <= 1e3 * f * scale + 1e-30), s
        assert np.all(vtr[s, m + 1:] == 0.0)
        assert np.max(np.abs(rr[lo:hi] - res)) <= 1e3 * f * (np.max(np.abs(ys[lo:hi])) + 1e-300)
        checked += 1
    assert checked > 120


@pytest.mark.parametrize("dtype,accum", [(torch.float32, "comp"), (torch.float64, "f64"),
                                         (torch.bfloat16, "comp")])
@pytest.mark.parametrize("tuning", [None, {"warp_max_len": 256, "chunk_len": 4096}])
def test_residuals_chebyshev_basis(L, dtype, accum, tuning):
    """Chebyshev-basis fits of degrees 1..8: f by Clenshaw's recurrence and
    (V^T r)_k = sum_i T_k(t_i) r_i, against the oracle's residuals of its own
    Chebyshev fit of the same stored points."""
    b = synth.ragged_batch(num_series=150, lmin=20, lmax=30000, mmin=1, mmax=8, seed=92,
                           a_range=(-5.0, 5.0), w_range=(1.0, 8.0))
    x = torch.from_numpy(b["x"]).to(dtype).cuda()
    y = torch.from_numpy(b["y"]).to(dtype).cuda()
    xs = x.double().cpu().numpy()
    ys = y.double().cpu().numpy()
    plan = L.BatchPlan(b["offsets"], 8, tuning=tuning, degree=b["degree"])
    fwd = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=8, accum=accum, plan=plan,
                        basis="chebyshev")
    out = L.residuals_batched(x, y, b["offsets"], b["degree"], fwd, want_r=True)
    sse = out["sse"].cpu().numpy()
    vtr = out["vtr"].cpu().numpy()
    rr = out["r"].double().cpu().numpy()
    tol = 1e-9 if dtype == torch.float64 else (1e-4 if dtype == torch.float32 else 1e-3)
    checked = 0
    for s in range(150):
        lo, hi = int(b["offsets"][s]), int(b["offsets"][s + 1])
        m = int(b["degree"][s])
        if L.status_names(fwd["status"][s: s + 1]) != ["ok"]:
            continue
        r = oracle.fit_general_interval(xs[lo:hi], ys[lo:hi], m, *b["interval"][s], fp32=accum != "f64",
                                        basis="chebyshev")
        assert r["status"] == "ok", s
        sse_ref, vtr_ref, res = oracle.residuals_general(xs[lo:hi], ys[lo:hi], r["Xb"], "chebyshev",
                                                         cs=(r["c"], r["s"]))
        t = r["s"] * (xs[lo:hi] - r["c"])
        scale = np.abs(np.polynomial.chebyshev.chebvander(t, m)).T @ np.abs(ys[lo:hi])
        assert abs(sse[s] - sse_ref) <= tol * sse_ref + 1e-30, (s, sse[s], sse_ref)
        f = 8 * m * (2.0 ** -53 if accum == "f64" else 2.0 ** -24)
        assert np.all(np.abs(vtr[s, : m + 1] - vtr_ref) <= 1e3 * f * scale + 1e-30), s
        assert np.all(vtr[s, m + 1:] == 0.0)
        assert np.max(np.abs(rr[lo:hi] - res)) <= 1e3 * f * (np.max(np.abs(ys[lo:hi])) + 1e-300)
        checked += 1
    assert checked > 120
    assert {int(m) for m in b["degree"]} == set(range(1, 9))


@pytest.mark.parametrize("basis", ["monomial", "chebyshev"])
def test_residuals_edge_series(L, basis):
    """Empty, too short, exactly interpolated, singular, non-finite, bad-interval
    and out-of-range-degree series (0, and 6 and 9 above m_max = 5): NaN SSE and
    V^T r for every failed fit (a whole NaN row for a degree outside 1..m_max),
    the oracle's values elsewhere."""
    rng = np.random.default_rng(93)
    lengths = np.array([0, 1, 2, 3, 6, 50, 5000, 70000, 0, 20, 20, 20, 33, 9000, 100, 200])
    b = synth.ragged_batch(lengths=lengths, seed=93, a_range=(-5.0, 5.0), w_range=(1.0, 8.0))
    b["degree"][:] = rng.integers(1, 6, lengths.size).astype(np.int32)
    b["degree"][3] = 3      # n = 3 < m + 1
    b["degree"][4] = 5      # n = m + 1: exact interpolation, SSE ~ 0
    b["degree"][12] = 0     # not fitted
    b["degree"][14] = 6     # above m_max = 5
    b["degree"][15] = 9     # above every kernel's degree
    off = b["offsets"]
    b["x"][off[9]: off[10]] = b["x"][off[9]]           # all-equal x: singular
    b["y"][off[10] + 4] = np.nan                      # non-finite
    b["interval"][11] = (2.0, 2.0)                    # bad interval
    x = torch.from_numpy(b["x"]).cuda()
    y = torch.from_numpy(b["y"]).cuda()
    for tuning in (None, {"warp_max_len": 8, "chunk_len": 1024}):
        plan = L.BatchPlan(b["offsets"], 5, tuning=tuning, degree=b["degree"])
        fwd = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, accum="comp", plan=plan,
                            basis=basis)
        out = L.residuals_batched(x, y, b["offsets"], b["degree"], fwd)
        st = L.status_names(fwd["status"])
        sse = out["sse"].cpu().numpy()
        vtr = out["vtr"].cpu().numpy()
        for s in (12, 14, 15):
            assert st[s] == "invalid_arg" and np.isnan(sse[s]) and np.all(np.isnan(vtr[s])), s
        good = 0
        for s in range(lengths.size):
            m = int(b["degree"][s])
            if s in (12, 14, 15):
                continue
            if st[s] != "ok":
                assert np.isnan(sse[s]) and np.all(np.isnan(vtr[s, : m + 1])) and np.all(vtr[s, m + 1:] == 0), s
                continue
            lo, hi = int(off[s]), int(off[s + 1])
            r = oracle.fit_general_interval(b["x"][lo:hi], b["y"][lo:hi], m, *b["interval"][s], fp32=True,
                                            basis=basis)
            if r["status"] != "ok":
                continue  # the 6-point degree-5 monomial system sits at the FP32 singularity threshold
            sse_ref, _, _ = oracle.residuals_general(b["x"][lo:hi], b["y"][lo:hi], r["Xb"], basis,
                                                     cs=(r["c"], r["s"]))
            ymax = float(np.max(np.abs(b["y"][lo:hi])))
            # absolute slack for the exactly interpolated series (SSE ~ 0): FP32 residuals
            assert abs(sse[s] - sse_ref) <= 1e-4 * sse_ref + (hi - lo) * (1e-4 * ymax) ** 2, (s, sse[s], sse_ref)
            good += 1
        assert st[0] == "n_too_small" and st[3] == "n_too_small" and st[8] == "n_too_small"
        assert st[9] == "singular" and st[10] == "nonfinite" and st[11] == "bad_interval"
        assert good >= (5 if basis == "chebyshev" else 4)  # the 6-point series is singular in monomials


def test_table5_sum_of_squared_errors(L):
    # Section III, Table I data, m = 3: the GPU's SSE of its own fit equals the
    # exact least-squares minimum and does not exceed the paper's printed value.
    rows, _ = read_golden("table1_sample.txt")
    x = np.array([float(r[0]) for r in rows])
    y = np.array([float(r[1]) for r in rows])
    rows5, _ = read_golden("table5_fitted.txt")
    sse_f = float(next(r[1] for r in rows5 if r[0] == "sse_f"))
    offsets = np.array([0, 6], dtype=np.int64)
    degree = np.array([3], dtype=np.int32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    fwd = L.fit_batched(xd, yd, offsets, degree, None, m_max=3, accum="f64")
    out = L.residuals_batched(xd, yd, offsets, degree, fwd, interval_given=False)
    gpu_sse = float(out["sse"].item())
    ref = oracle.fit(x, y, 3)
    assert abs(gpu_sse - oracle.sse(ref["X"], x, y)) <= 1e-8 * gpu_sse
    assert gpu_sse <= sse_f
    assert np.allclose(fwd["X"][0].cpu().numpy(), ref["X"], rtol=1e-8)


def test_full_size_residuals_sampled(L):
    """The 65,536-series batch at the benchmark's size: SSE of sampled series
    against the oracle's residuals of its own fit."""
    b = synth.ragged_batch()
    x = torch.from_numpy(b["x"]).cuda()
    y = torch.from_numpy(b["y"]).cuda()
    fwd = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, accum="comp")
    out = L.residuals_batched(x, y, b["offsets"], b["degree"], fwd)
    sse = out["sse"].cpu().numpy()
    rng = np.random.default_rng(92)
    for s in rng.choice(len(b["degree"]), 200, replace=False):
        lo, hi = int(b["offsets"][s]), int(b["offsets"][s + 1])
        xs = b["x"][lo:hi].astype(np.float64)
        ys = b["y"][lo:hi].astype(np.float64)
        _, sse_ref, _, _, _ = _ref(xs, ys, int(b["degree"][s]), *b["interval"][s], fp32=True)
        assert abs(sse[s] - sse_ref) <= 1e-4 * sse_ref + 1e-30, (s, sse[s], sse_ref)
