"""Parity of the single-series CUDA path (lsefit_powersums + lsefit_solve) with the oracle.

Tolerances (relative 2-norm errors of the mapped-basis coefficients Xt; the
policy and its reasons are in tests/gates.py):
  * FP64 accumulation: 1e-6;
  * compensated FP32 on x mapped to [-1, 1]: 1e-5 at every degree up to 8
    (measured at most 3.1e-7 at m = 8, cond(A) = 3e5);
  * every ok result also passes the backward-error gate of its accumulation
    (the GPU's Xt in the oracle's own normal equations), which does not
    depend on cond(A).
Where the oracle's own result is ill-determined (cond(A) * eps64 not small)
only the mapped basis is compared.
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


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _hankel(S, m):
    return np.array([[S[j + k] for k in range(m + 1)] for j in range(m + 1)])


def _bf16_dev(bits):
    return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()


# --- FP64: the plain method on the FP64 single-series workload -------------------------

@pytest.mark.parametrize("m", [1, 2, 3])
def test_fp64_single_series(L, m):
    d = synth.single_fp64()
    ref = oracle.fit(d["x"], d["y"], m)
    out = L.fit(_dev(d["x"]), _dev(d["y"]), m, accum="f64")
    assert L.status_names(out["status"]) == ["ok"]
    X = out["X"].cpu().numpy()
    assert _rel(X, ref["X"]) <= 1e-6
    sums = out["sums"].cpu().numpy()
    np.testing.assert_allclose(sums[: 2 * m + 1], ref["S"], rtol=1e-12)
    np.testing.assert_allclose(sums[2 * m + 1:], ref["T"], rtol=1e-12)


# --- bit-exact power sums on small integers -----------------------------------------

@pytest.mark.parametrize("accum,dtype,n", [("f64", torch.float64, 100_003), ("f64", torch.float32, 70_001),
                                           ("comp", torch.float32, 100_003), ("comp", torch.float32, 3001),
                                           ("naive", torch.float32, 1000), ("comp", torch.bfloat16, 50_001)])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_powersums_bit_exact_int(L, accum, dtype, n, m):
    rng = np.random.default_rng(7000 + n + m)
    xi = rng.integers(-8, 9, n)
    yi = rng.integers(-100, 101, n)
    x = _dev(xi.astype(np.float64), dtype)
    y = _dev(yi.astype(np.float64), dtype)
    sums, mp, st = L.powersums(x, y, m, accum)
    got = sums.cpu().numpy()
    x64 = xi.astype(np.int64)
    for k in range(2 * m + 1):
        assert got[k] == float(int(np.sum(x64 ** k))), (k, got[k])
    for k in range(m + 1):
        assert got[2 * m + 1 + k] == float(int(np.sum(x64 ** k * yi))), (k,)
    assert int(st.item()) == L.OK


# --- FP32 on [-1, 1] (the long-series workload, smaller n) -----------------------------

@pytest.mark.parametrize("accum", ["comp", "naive", "f64"])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_fp32_unit_interval(L, accum, m):
    d = synth.single_large(n=(1 << 20) + 13, m=m, seed=42 + m)
    ref = oracle.fit(d["x"], d["y"], m)
    out = L.fit(_dev(d["x"]), _dev(d["y"]), m, accum=accum)
    assert L.status_names(out["status"]) == ["ok"]
    tol = 1e-6 if accum == "f64" else 1e-5
    assert _rel(out["Xt"].cpu().numpy(), ref["Xt"]) <= tol
    assert _rel(out["X"].cpu().numpy(), ref["X"]) <= tol


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("accum", ["comp", "f64"])
def test_fp32_mapped_unscaled_interval(L, m, accum):
    # precision workload shape (x on [0, 1000], mapped), at 2^20 points
    d = synth.precision(n=1 << 20, m=m)
    lo, hi = d["interval"]
    fp32_map = accum != "f64"
    ref = oracle.fit_interval(d["x"], d["y"], m, lo, hi, fp32=fp32_map)
    out = L.fit(_dev(d["x"]), _dev(d["y"]), m, accum=accum, interval=(lo, hi))
    assert L.status_names(out["status"]) == ["ok"]
    mp = out["map"].cpu().numpy()
    assert mp[0] == ref["c"] and mp[1] == ref["s"]
    tol = 1e-6 if accum == "f64" else 1e-5
    Xt = out["Xt"].cpu().numpy()
    assert _rel(Xt, ref["Xt"]) <= tol, tol
    A = _hankel(ref["S"], m)
    assert gates.backward_error(A, ref["T"], Xt) <= gates.backward_gate(accum, d["x"].size)


@pytest.mark.parametrize("m", [1, 3, 5])
def test_bf16_storage(L, m):
    d = synth.precision(n=1 << 18, m=m, lo=-1.0, hi=1.0)
    xb, yb = d["x_bf16"], d["y_bf16"]
    x64 = synth.from_bf16_bits(xb).astype(np.float64)
    y64 = synth.from_bf16_bits(yb).astype(np.float64)
    ref = oracle.fit_interval(x64, y64, m, -1.0, 1.0, fp32=True)
    for accum in ("comp", "f64"):
        out = L.fit(_bf16_dev(xb), _bf16_dev(yb), m, accum=accum, interval=(-1.0, 1.0))
        assert L.status_names(out["status"]) == ["ok"]
        Xt = out["Xt"].cpu().numpy()
        # BF16 storage, m <= 5: measured at most 3.9e-7 (compensated) on the 2^24 grid
        assert _rel(Xt, ref["Xt"]) <= (1e-6 if accum == "f64" else 1e-5)
        assert gates.backward_error(_hankel(ref["S"], m), ref["T"], Xt) <= gates.backward_gate(accum, xb.size)


# --- ragged sizes, alignment and tails ---------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 7, 8, 9, 31, 33, 255, 257, 1000, 4097, 65537, 300_001])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
def test_sizes_and_tails(L, n, dtype):
    m = 2
    d = synth.small_series(n + 3, seed=n, m=m, dtype=np.float64)
    xs = torch.from_numpy(d["x"]).to(dtype)
    ys = torch.from_numpy(d["y"]).to(dtype)
    accum = "f64" if dtype == torch.float64 else "comp"
    # offsets (0, 0): aligned; (1, 1): same misalignment; (1, 2): different misalignment
    for ox, oy in [(0, 0), (1, 1), (1, 2), (3, 3)]:
        x = xs.cuda()[ox: ox + n]
        y = ys.cuda()[oy: oy + n]
        sums, mp, st = L.powersums(x, y, m, accum)
        xr = x.double().cpu().numpy()
        yr = y.double().cpu().numpy()
        S, T = oracle.powersums(xr, yr, m)
        got = sums.cpu().numpy()
        scale_S = np.array([np.sum(np.abs(xr) ** k) for k in range(2 * m + 1)])
        scale_T = np.array([np.sum(np.abs(xr) ** k * np.abs(yr)) for k in range(m + 1)])
        tol = 1e-12 if accum == "f64" else 8 * m * EPS32
        assert np.all(np.abs(got[: 2 * m + 1] - S) <= tol * scale_S + 1e-300), (ox, oy)
        assert np.all(np.abs(got[2 * m + 1:] - T) <= tol * scale_T + 1e-300), (ox, oy)
        assert got[0] == n


# --- statuses ---------------------------------------------------------------------

def test_statuses(L):
    f32 = torch.float32
    out = L.fit(_dev(np.array([1.0, 2.0]), f32), _dev(np.array([1.0, 2.0]), f32), 2)
    assert L.status_names(out["status"]) == ["n_too_small"]
    assert torch.isnan(out["X"]).all()
    out = L.fit(_dev(np.full(100, 2.0), f32), _dev(np.arange(100.0), f32), 1)
    assert L.status_names(out["status"]) == ["singular"]
    y = np.arange(100.0)
    y[37] = np.nan
    out = L.fit(_dev(np.linspace(-1, 1, 100), f32), _dev(y, f32), 2)
    assert L.status_names(out["status"]) == ["nonfinite"]
    out = L.fit(_dev(np.linspace(-1, 1, 100), f32), _dev(np.arange(100.0), f32), 2,
                interval=(1.0, 1.0))
    assert L.status_names(out["status"]) == ["bad_interval"]
    assert torch.isnan(out["sums"]).all() and torch.isnan(out["map"]).all()
    # FP32 overflow of the unscaled high powers: x ~ 1000, m = 8 -> x^16 = 1e48
    x = np.linspace(0.0, 1000.0, 4096)
    out = L.fit(_dev(x, f32), _dev(np.ones_like(x), f32), 8, accum="comp")
    assert L.status_names(out["status"]) == ["nonfinite"]
    # the same data mapped to [-1, 1] is fine
    out = L.fit(_dev(x, f32), _dev(np.sin(x / 100), f32), 8, accum="comp", interval=(0.0, 1000.0))
    assert L.status_names(out["status"]) == ["ok"]


def test_invalid_arguments(L):
    x = torch.zeros(10, device="cuda")
    with pytest.raises(ValueError):  # rejected by the binding before the call
        L.powersums(x, x, 9)
    sums = torch.empty(32, dtype=torch.float64, device="cuda")
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    from paper_1512_08017_gb300 import lsefit as B
    rc = B.lib.lsefit_powersums(B._ptr(x), B._ptr(x), 10, B.F32, 9, 1, None, B._ptr(sums), None, None,
                                B._ptr(ws), ws.numel(), None)
    assert rc == L.ERR_INVALID_ARG
    with pytest.raises(L.LsefitError):
        L.powersums(x.double(), x.double(), 2, accum="comp")  # F64 data needs F64 accumulation


# --- determinism and nested degrees ------------------------------------------------------

def test_deterministic(L):
    d = synth.single_large(n=3_000_017, m=3, seed=5)
    x, y = _dev(d["x"]), _dev(d["y"])
    a = L.powersums(x, y, 3, "comp")[0].clone()
    for _ in range(3):
        b = L.powersums(x, y, 3, "comp")[0]
        assert torch.equal(a, b)


def test_lower_degrees_from_one_pass(L):
    d = synth.single_large(n=1 << 20, m=3, seed=9)
    x, y = _dev(d["x"]), _dev(d["y"])
    sums, mp, _ = L.powersums(x, y, 3, "comp")
    for m in (1, 2):
        X, Xt, st = L.solve(sums, m, 3, mp)
        ref = oracle.fit(d["x"], d["y"], m)
        assert L.status_names(st) == ["ok"]
        assert _rel(X.cpu().numpy(), ref["X"]) <= 1e-5


def test_mapped_host_memory(L):
    # points in pinned host memory are streamed by the kernel directly
    d = synth.single_large(n=(1 << 18) + 5, m=3, seed=12)
    x = torch.from_numpy(d["x"]).pin_memory()
    y = torch.from_numpy(d["y"]).pin_memory()
    out = L.fit(x, y, 3, accum="comp")
    ref = oracle.fit(d["x"], d["y"], 3)
    assert L.status_names(out["status"]) == ["ok"]
    assert _rel(out["X"].cpu().numpy(), ref["X"]) <= 1e-5


# --- fused single-launch fit of several degrees (lsefit_fit) ------------------------------

@pytest.mark.parametrize("m,m_lo", [(3, 1), (5, 2), (8, 8), (1, 1)])
def test_fused_fit_degrees(L, m, m_lo):
    d = synth.single_large(n=(1 << 20) + 3, m=min(m, 4), seed=60 + m)
    x, y = _dev(d["x"]), _dev(d["y"])
    out = L.fit_degrees(x, y, m, m_lo, accum="comp", interval=(-1.0, 1.0))
    assert L.status_names(out["status"]) == ["ok"] * (m - m_lo + 1)
    X = out["X"].cpu().numpy()
    Xt = out["Xt"].cpu().numpy()
    for r, deg in enumerate(range(m_lo, m + 1)):
        ref = oracle.fit_interval(d["x"], d["y"], deg, -1.0, 1.0, fp32=True)
        assert _rel(Xt[r, : deg + 1], ref["Xt"]) <= 1e-5, deg
        assert gates.backward_error(_hankel(ref["S"], deg), ref["T"], Xt[r, : deg + 1]) <= gates.BACKWARD["comp"]
        assert np.all(X[r, deg + 1:] == 0.0)
        # same as the two-launch path
        X2, Xt2, st2 = L.solve(out["sums"], deg, m, out["map"])
        assert _rel(Xt[r, : deg + 1], Xt2.cpu().numpy()) <= 1e-12


def test_fused_fit_statuses(L):
    f32 = torch.float32
    out = L.fit_degrees(_dev(np.linspace(-1, 1, 3), f32), _dev(np.ones(3), f32), 4, 1)
    assert L.status_names(out["status"]) == ["ok", "ok", "n_too_small", "n_too_small"]
    out = L.fit_degrees(_dev(np.linspace(-1, 1, 30), f32), _dev(np.ones(30), f32), 2, 1, interval=(3.0, 1.0))
    assert L.status_names(out["status"]) == ["bad_interval", "bad_interval"]


# --- alternative solver: Cholesky ---------------------------------------------------------

@pytest.mark.parametrize("m", [1, 3, 5, 8])
def test_cholesky_solver(L, m):
    d = synth.precision(n=1 << 18, m=min(m, 5))
    lo, hi = d["interval"]
    sums, mp, _ = L.powersums(_dev(d["x"]), _dev(d["y"]), m, "comp", (lo, hi))
    Xg, Xtg, stg = L.solve(sums, m, m, mp, "comp")
    Xc, Xtc, stc = L.solve(sums, m, m, mp, "comp", method="cholesky")
    assert L.status_names(stc) == ["ok"] and L.status_names(stg) == ["ok"]
    S = sums.cpu().numpy()
    st, Xo = oracle.solve_cholesky(S[: 2 * m + 1], S[2 * m + 1:], m, eps=oracle.EPS32)
    assert st == "ok"
    cond = np.linalg.cond(_hankel(S[: 2 * m + 1], m))
    assert _rel(Xtc.cpu().numpy(), Xo) <= 1e2 * cond * 2.0 ** -52
    assert _rel(Xtc.cpu().numpy(), Xtg.cpu().numpy()) <= 1e2 * cond * 2.0 ** -52


def test_cholesky_statuses(L):
    f32 = torch.float32
    sums, mp, _ = L.powersums(_dev(np.full(50, 2.0), f32), _dev(np.arange(50.0), f32), 2, "comp")
    X, Xt, st = L.solve(sums, 2, 2, mp, "comp", method="cholesky")
    assert L.status_names(st) == ["singular"] and torch.isnan(X).all()


@pytest.mark.parametrize("m", [1, 2, 3])
def test_fp64_mapped_coefficients(L, m):
    """FP64 data on [0, 10] mapped to [-1, 1]: the un-mapped x-basis coefficients
    match the oracle's (the un-map is well conditioned for c = 5, s = 0.2)."""
    d = synth.single_fp64()
    ref = oracle.fit_interval(d["x"], d["y"], m, 0.0, 10.0, fp32=False)
    out = L.fit(_dev(d["x"]), _dev(d["y"]), m, accum="f64", interval=(0.0, 10.0))
    assert L.status_names(out["status"]) == ["ok"]
    assert _rel(out["Xt"].cpu().numpy(), ref["Xt"]) <= 1e-9
    assert _rel(out["X"].cpu().numpy(), ref["X"]) <= 1e-9


# --- the benchmark's own call at its full size ----------------------------------------------

def test_full_size_bench_call(L):
    """The call bench.py times, on its workload: fit_degrees(x, y, 3, 1, "comp") on the
    2^28-point FP32 series (x on [-1, 1], no interval), in the launch configuration of
    that size (304 blocks, ~860 grid-stride rounds per thread).  Every degree's X and Xt
    against the oracle's fit of the same stored points, the saved sums within the
    compensated-FP32 summation bound, and a second call bit-identical to the first."""
    n = 1 << 28
    d = synth.single_large(n=n, m=3, seed=synth.SEED_SINGLE_LARGE)
    x, y = _dev(d["x"]), _dev(d["y"])
    out = L.fit_degrees(x, y, 3, 1, "comp")
    torch.cuda.synchronize()
    assert L.status_names(out["status"]) == ["ok"] * 3
    X = out["X"].cpu().numpy()
    Xt = out["Xt"].cpu().numpy()
    sums = out["sums"].cpu().numpy()
    again = L.fit_degrees(x, y, 3, 1, "comp")
    assert torch.equal(again["X"], out["X"]) and torch.equal(again["sums"], out["sums"])
    del x, y, again
    x64 = d["x"].astype(np.float64)
    y64 = d["y"].astype(np.float64)
    ref = oracle.fit(x64, y64, 3, eps=oracle.EPS32)
    assert ref["status"] == "ok"
    S, T = ref["S"], ref["T"]
    for r, deg in enumerate((1, 2, 3)):
        st, Xo = oracle.solve(S[: 2 * deg + 1], T[: deg + 1], deg, eps=oracle.EPS32)
        assert st == "ok"
        assert _rel(Xt[r, : deg + 1], Xo) <= 1e-5, deg
        assert _rel(X[r, : deg + 1], Xo) <= 1e-5, deg  # no interval: X = Xt
        assert np.all(X[r, deg + 1:] == 0.0)
        assert gates.backward_error(_hankel(S, deg), T[: deg + 1], Xt[r, : deg + 1]) <= gates.BACKWARD["comp"]
    # sums: S_0 exact; the others within the bound of the compensated FP32 pass
    # (batches of 8 points per packed lane at degree 3), scaled by sum |x|^k (|y|)
    Sa, Ta = oracle.powersums(np.abs(x64), np.abs(y64), 3)
    assert sums[0] == n
    for k in range(1, 7):
        assert abs(sums[k] - S[k]) <= gates.sums_bound(k, Sa[k], batch=8), k
    for k in range(4):
        assert abs(sums[7 + k] - T[k]) <= gates.sums_bound(k + 1, Ta[k], batch=8), k


# --- the eliminations' reciprocal -------------------------------------------------------

def test_reciprocal_within_two_ulp_of_ieee_division(L):
    """The pivots' reciprocal (Newton-Raphson refinement of an FP32 seed) against
    IEEE division on the GPU: within 2 ulp over magnitudes from 2^-1021 to 2^1021,
    both signs; zero, infinities and NaN as IEEE division gives them."""
    from paper_1512_08017_gb300 import lsefit as B
    rng = np.random.default_rng(123)
    mant = rng.uniform(1.0, 2.0, 200_000)
    ex = rng.integers(-1021, 1021, mant.size)
    a = np.ldexp(mant, ex) * rng.choice([-1.0, 1.0], mant.size)
    a = np.concatenate([a, [1.0, 2.0, 1.5, np.nextafter(2.0, 0.0), 3.0, 0.1, -7.0, 1e300, -1e-300]])
    ad = torch.from_numpy(a).cuda()
    out = torch.empty_like(ad)
    assert B.lib.lsefit_check_reciprocal(B._ptr(ad), B._ptr(out), a.size, None) == B.OK
    ref = (1.0 / ad).cpu().numpy()
    got = out.cpu().numpy()
    ulp = np.spacing(np.abs(ref))
    assert np.max(np.abs(got - ref) / ulp) <= 2.0
    special = torch.tensor([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 2.0 ** 1023], dtype=torch.float64).cuda()
    so = torch.empty_like(special)
    assert B.lib.lsefit_check_reciprocal(B._ptr(special), B._ptr(so), special.numel(), None) == B.OK
    sr = (1.0 / special).cpu().numpy()
    sg = so.cpu().numpy()
    assert np.array_equal(np.isnan(sg), np.isnan(sr))
    fin = ~np.isnan(sr)
    assert np.array_equal(sg[fin], sr[fin])
