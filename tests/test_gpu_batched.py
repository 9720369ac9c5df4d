"""Parity of the batched ragged CUDA path (lsefit_fit_batched) with the oracle, series by series.

Each series is compared with the oracle's fit of the same stored points on
the same map (FP32-rounded constants for FP32 arithmetic, FP64 otherwise).
Statuses must match the oracle's exactly.  Coefficients follow the policy of
tests/gates.py: the mapped-basis Xt within max(1e-6 | 1e-5, cond(A_t) eps 4m)
wherever that bound is at most 1e-3 (reported beyond, where the data leave
the coefficients undetermined), and always within the backward-error gate of
the accumulation.  Saved sums within the summation bound of the accumulation.
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


def _hankel(S, m):
    return np.array([[S[j + k] for k in range(m + 1)] for j in range(m + 1)])


def check_batch(L, b, res, accum, stored_x=None, stored_y=None, series=None, fp32_map=None, sums_every=1,
                stats=None):
    """Check series `series` (all by default) against the oracle; the saved sums of
    every sums_every-th checked series.  stats (a dict) collects the largest
    forward and backward errors and the count of forward-reported series."""
    if fp32_map is None:
        fp32_map = accum != "f64"  # FP64 arithmetic maps with FP64 constants
    X = res["X"].cpu().numpy()
    Xt = res["Xt"].cpu().numpy()
    st = res["status"].cpu().numpy()
    sums = res["sums"].cpu().numpy()
    mp = res["map"].cpu().numpy()
    xs = stored_x if stored_x is not None else b["x"].astype(np.float64)
    ys = stored_y if stored_y is not None else b["y"].astype(np.float64)
    S = len(b["offsets"]) - 1
    checked = 0
    for s in (range(S) if series is None else series):
        lo, hi = int(b["offsets"][s]), int(b["offsets"][s + 1])
        m = int(b["degree"][s])
        if b.get("interval") is not None:
            r = oracle.fit_interval(xs[lo:hi], ys[lo:hi], m, *b["interval"][s], fp32=fp32_map)
        else:
            r = oracle.fit(xs[lo:hi], ys[lo:hi], m, eps=oracle.EPS64 if accum == "f64" else oracle.EPS32)
        got = L.STATUS_NAMES.get(int(st[s]), str(st[s]))
        assert got == r["status"], (s, got, r["status"], hi - lo, m)
        if r["status"] != "ok":
            assert np.all(np.isnan(X[s, : m + 1]))
            continue
        if b.get("interval") is not None:
            assert mp[s, 0] == r["c"] and mp[s, 1] == r["s"], s
        A = gates.hankel(r["S"], m)
        try:
            ef, tol, eta = gates.check_coefficients(Xt[s, : m + 1], r["Xt"], A, r["T"], accum, m, n=hi - lo)
        except AssertionError as exc:
            raise AssertionError((s, hi - lo) + tuple(exc.args)) from None
        if stats is not None:
            stats["forward_max"] = max(stats.get("forward_max", 0.0), ef if tol is not None else 0.0)
            stats["backward_max"] = max(stats.get("backward_max", 0.0), eta)
            stats["reported"] = stats.get("reported", 0) + (tol is None)
        assert np.all(X[s, m + 1:] == 0.0) and np.all(Xt[s, m + 1:] == 0.0)
        if b.get("interval") is not None:
            # the x-basis coefficients (the un-map of Xt) give the same polynomial: values
            # across the interval agree up to the Xt tolerance plus the rounding of an
            # x-basis evaluation (relative to the size of its terms)
            xx = np.linspace(b["interval"][s][0], b["interval"][s][1], 5)
            tt = r["s"] * (xx - r["c"])
            pw = np.arange(m + 1)
            f_ref = (r["Xt"][None, :] * tt[:, None] ** pw).sum(axis=1)
            terms = X[s, : m + 1][None, :] * xx[:, None] ** pw
            if tol is not None:
                slack = 2 * tol * np.linalg.norm(r["Xt"]) * (m + 1) + 1e-11 * np.abs(terms).sum(axis=1)
                assert np.all(np.abs(terms.sum(axis=1) - f_ref) <= slack), (s, m)
        # saved sums: S_0 exact, the others within the summation bound of the
        # accumulation, scaled by sum |t|^k (|y|) of the same mapped points
        assert sums[s, 0] == hi - lo
        if checked % sums_every == 0:
            t = xs[lo:hi] if b.get("interval") is None else r["s"] * (xs[lo:hi] - r["c"])
            Sa, Ta = oracle.powersums(np.abs(t), np.abs(ys[lo:hi]), m)
            lane = -(-(hi - lo) // 32)
            for k in range(1, 2 * m + 1):
                assert abs(sums[s, k] - r["S"][k]) <= gates.sums_bound_for(accum, k, Sa[k], lane), (s, k)
            for k in range(m + 1):
                assert abs(sums[s, 2 * m + 1 + k] - r["T"][k]) <= \
                    gates.sums_bound_for(accum, k + 1, Ta[k], lane), (s, "T", k)
        checked += 1
    return checked


def _run(L, b, accum="comp", dtype=torch.float32, tuning=None, m_max=5, with_interval=True):
    dev = torch.device("cuda")
    x = torch.from_numpy(b["x"]).to(dev).to(dtype)
    y = torch.from_numpy(b["y"]).to(dev).to(dtype)
    plan = L.BatchPlan(b["offsets"], m_max, tuning=tuning, degree=b["degree"])
    res = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"] if with_interval else None,
                        m_max=m_max, accum=accum, plan=plan)
    torch.cuda.synchronize()
    return x, y, res, plan


@pytest.mark.parametrize("accum", ["comp", "naive", "f64"])
def test_ragged_all_warp_tasks(L, accum):
    b = synth.ragged_batch(num_series=300, lmin=1, lmax=70000, seed=44)
    _, _, res, plan = _run(L, b, accum, tuning={"warp_max_len": 1 << 20})
    assert plan.plan.n_block_tasks == 0
    assert check_batch(L, b, res, accum) > 250


@pytest.mark.parametrize("accum", ["comp", "naive", "f64"])
def test_ragged_mixed_degrees(L, accum):
    b = synth.ragged_batch(num_series=400, lmin=16, lmax=40000, seed=31)
    _, _, res, plan = _run(L, b, accum, tuning={"warp_max_len": 8192, "chunk_len": 65536})
    assert plan.plan.n_block_tasks > 0 and plan.plan.n_warp_tasks > 0
    assert check_batch(L, b, res, accum) > 350


@pytest.mark.parametrize("tuning", [{"warp_max_len": 64, "chunk_len": 1024},
                                    {"warp_max_len": 1 << 20},
                                    {"warp_max_len": 16, "chunk_len": 4096, "blocks_per_sm": 1},
                                    {"warp_max_len": 1 << 20, "schedule": 1, "task_order": 1},
                                    {"warp_max_len": 1 << 20, "schedule": 1, "task_order": 2},
                                    {"warp_max_len": 1 << 20, "schedule": 2},
                                    {"warp_max_len": 64, "chunk_len": 1024, "schedule": 2}])
def test_schedules_agree(L, tuning):
    b = synth.ragged_batch(num_series=300, lmin=1, lmax=30000, seed=32)
    _, _, res, plan = _run(L, b, "comp", tuning=tuning)
    if tuning.get("chunk_len") == 1024:
        assert plan.plan.n_split_series > 0
    assert check_batch(L, b, res, "comp") > 250


def test_workspace_shared_by_layouts(L):
    # one cached workspace serves plans of different layouts in turn
    b1 = synth.ragged_batch(num_series=50, lmin=16, lmax=3000, seed=42)
    b2 = synth.ragged_batch(num_series=400, lmin=16, lmax=30000, seed=43)
    for b, tuning in ((b1, None), (b2, {"warp_max_len": 64, "chunk_len": 1024}), (b1, None),
                      (b2, {"warp_max_len": 512, "chunk_len": 2048})):
        _, _, res, _ = _run(L, b, "comp", tuning=tuning)
        check_batch(L, b, res, "comp")


def test_deterministic_and_reusable(L):
    b = synth.ragged_batch(num_series=500, lmin=16, lmax=20000, seed=33)
    x, y, res, plan = _run(L, b, "comp", tuning={"warp_max_len": 512, "chunk_len": 2048})
    X0 = res["X"].clone()
    assert torch.isfinite(X0).all()
    for _ in range(3):
        r2 = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, accum="comp", plan=plan)
        assert torch.equal(r2["X"], X0)


def test_edge_series(L):
    rng = np.random.default_rng(34)
    lengths = np.array([0, 1, 2, 3, 6, 50, 5000, 70000, 0, 20, 20, 20, 33, 9000])
    b = synth.ragged_batch(lengths=lengths, seed=34)
    b["degree"][:] = rng.integers(1, 6, lengths.size).astype(np.int32)
    b["degree"][3] = 3      # n = 3 < m + 1
    b["degree"][4] = 5      # n = 6 = m + 1: exact interpolation
    off = b["offsets"]
    b["x"][off[9]: off[10]] = b["x"][off[9]]           # all-equal x: singular
    b["y"][off[10] + 4] = np.nan                      # non-finite
    b["interval"][11] = (2.0, 2.0)                    # bad interval
    for tuning in (None, {"warp_max_len": 8, "chunk_len": 1024}):
        _, _, res, _ = _run(L, b, "comp", tuning=tuning)
        st = L.status_names(res["status"])
        assert st[0] == "n_too_small" and st[3] == "n_too_small" and st[8] == "n_too_small"
        assert st[9] == "singular" and st[10] == "nonfinite" and st[11] == "bad_interval"
        assert check_batch(L, b, res, "comp") >= 5


@pytest.mark.parametrize("tuning", [None, {"warp_max_len": 1 << 20, "schedule": 1},
                                    {"warp_max_len": 1 << 20, "schedule": 2},
                                    {"warp_max_len": 256, "chunk_len": 1024}])
def test_invalid_degrees(L, tuning):
    """Degrees outside 1..m_max leave a NaN row and the invalid-argument status;
    the other series of the batch are fitted as usual."""
    b = synth.ragged_batch(num_series=200, lmin=16, lmax=5000, seed=39)
    bad = {3: 0, 17: -2, 40: 6, 41: 9, 100: 1000}
    for s, m in bad.items():
        b["degree"][s] = m
    _, _, res, _ = _run(L, b, "comp", tuning=tuning)
    st = res["status"].cpu().numpy()
    X = res["X"].cpu().numpy()
    for s in bad:
        assert L.STATUS_NAMES[int(st[s])] == "invalid_arg" and np.all(np.isnan(X[s])), s
    good = [s for s in range(200) if s not in bad]
    assert check_batch(L, b, res, "comp", series=good) > 180


def test_high_degrees(L):
    b = synth.ragged_batch(num_series=120, lmin=64, lmax=30000, mmin=1, mmax=8, seed=35,
                           a_range=(-1.0, 1.0), w_range=(1.0, 3.0))
    _, _, res, _ = _run(L, b, "comp", m_max=8, tuning={"warp_max_len": 2048, "chunk_len": 8192})
    assert check_batch(L, b, res, "comp") > 100


def test_fp64_storage(L):
    b = synth.ragged_batch(num_series=200, lmin=16, lmax=20000, seed=36)
    b["x"] = b["x"].astype(np.float64)
    b["y"] = b["y"].astype(np.float64)
    _, _, res, _ = _run(L, b, "f64", dtype=torch.float64)
    assert check_batch(L, b, res, "f64", fp32_map=False) > 180


def test_bf16_storage(L):
    b = synth.ragged_batch(num_series=200, lmin=16, lmax=20000, seed=37, a_range=(-2.0, 2.0),
                           w_range=(1.0, 4.0))
    xb = synth.from_bf16_bits(synth.to_bf16_bits(b["x"])).astype(np.float64)
    yb = synth.from_bf16_bits(synth.to_bf16_bits(b["y"])).astype(np.float64)
    _, _, res, _ = _run(L, b, "comp", dtype=torch.bfloat16)
    assert check_batch(L, b, res, "comp", stored_x=xb, stored_y=yb) > 150


def test_no_interval(L):
    b = synth.ragged_batch(num_series=200, lmin=16, lmax=20000, seed=38, a_range=(-1.0, -0.5),
                           w_range=(0.5, 1.0))
    _, _, res, _ = _run(L, b, "comp", with_interval=False)
    bb = dict(b)
    bb["interval"] = None
    assert check_batch(L, bb, res, "comp") > 100


def test_matches_single_series_path(L):
    # the batched result of a series equals the single-series path within rounding
    b = synth.ragged_batch(num_series=40, lmin=1000, lmax=200000, seed=39)
    x, y, res, _ = _run(L, b, "comp")
    for s in range(0, 40, 7):
        lo, hi = int(b["offsets"][s]), int(b["offsets"][s + 1])
        m = int(b["degree"][s])
        one = L.fit(x[lo:hi], y[lo:hi], m, accum="comp", interval=tuple(b["interval"][s]))
        a = res["Xt"][s, : m + 1].cpu().numpy()
        c = one["Xt"].cpu().numpy()
        assert np.linalg.norm(a - c) / np.linalg.norm(c) <= 1e-5


def test_cuda_graph_replay(L):
    b = synth.ragged_batch(num_series=300, lmin=16, lmax=20000, seed=40)
    x, y, res, plan = _run(L, b, "comp")
    ref = res["X"].clone()
    out = {k: torch.empty_like(v) for k, v in res.items() if isinstance(v, torch.Tensor)}
    off_d = torch.from_numpy(b["offsets"]).cuda()
    deg_d = torch.from_numpy(b["degree"]).cuda()
    iv_d = torch.from_numpy(b["interval"]).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        L.fit_batched(x, y, off_d, deg_d, iv_d, m_max=5, accum="comp", plan=plan, out=out)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        L.fit_batched(x, y, off_d, deg_d, iv_d, m_max=5, accum="comp", plan=plan, out=out)
    for _ in range(3):
        out["X"].zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(torch.nan_to_num(out["X"]), torch.nan_to_num(ref))


def test_full_size_ragged_all_series(L):
    """The 65,536-series workload at the launch configuration the benchmark times
    (the default plan: degree classes, warp tasks up to 65,536 points): every
    series' status and coefficients against the oracle, the saved sums of one
    series in 16."""
    b = synth.ragged_batch()
    _, _, res, plan = _run(L, b, "comp")
    st = res["status"].cpu().numpy()
    assert np.all(st == 0)
    stats = {}
    S = len(b["degree"])
    assert check_batch(L, b, res, "comp", sums_every=16, stats=stats) == S
    print(f"ragged 65536: forward max {stats['forward_max']:.3g}, backward max {stats['backward_max']:.3g}, "
          f"forward reported {stats['reported']}")


# --- the Chebyshev basis in the batched kernel ----------------------------------------

def _check_cheb(L, b, res, accum, xs, ys, series=None):
    """Per series: Chebyshev coefficients (Xt) against the oracle's fit in the same
    basis, statuses equal, and the x-basis polynomial X gives the same values."""
    X = res["X"].cpu().numpy()
    Xt = res["Xt"].cpu().numpy()
    st = res["status"].cpu().numpy()
    checked = 0
    for s in (range(len(b["degree"])) if series is None else series):
        lo, hi = int(b["offsets"][s]), int(b["offsets"][s + 1])
        m = int(b["degree"][s])
        r = oracle.fit_general_interval(xs[lo:hi], ys[lo:hi], m, *b["interval"][s], fp32=accum != "f64",
                                        basis="chebyshev")
        got = L.STATUS_NAMES.get(int(st[s]), str(st[s]))
        assert got == r["status"], (s, got, r["status"], hi - lo, m)
        if r["status"] != "ok":
            continue
        ef, tol, eta = gates.check_coefficients(Xt[s, : m + 1], r["Xb"], r["G"], r["b"], accum, m, n=hi - lo)
        if tol is None:
            checked += 1
            continue
        xx = np.linspace(b["interval"][s][0], b["interval"][s][1], 5)
        f_ref = np.polynomial.chebyshev.chebval(r["s"] * (xx - r["c"]), r["Xb"])
        terms = X[s, : m + 1][None, :] * xx[:, None] ** np.arange(m + 1)
        slack = 2 * tol * np.abs(r["Xb"]).sum() + 1e-11 * np.abs(terms).sum(axis=1)
        assert np.all(np.abs(terms.sum(axis=1) - f_ref) <= slack), (s, m)
        checked += 1
    return checked


@pytest.mark.parametrize("dtype,accum", [(torch.float32, "comp"), (torch.bfloat16, "comp"),
                                         (torch.float32, "f64"), (torch.float64, "f64")])
@pytest.mark.parametrize("tuning", [None, {"warp_max_len": 512, "chunk_len": 2048}])
def test_chebyshev_basis(L, dtype, accum, tuning):
    b = synth.ragged_batch(num_series=300, lmin=16, lmax=30000, seed=44)
    b["degree"][5] = 0  # not fitted: status and NaN row
    x = torch.from_numpy(b["x"]).to(dtype).cuda()
    y = torch.from_numpy(b["y"]).to(dtype).cuda()
    plan = L.BatchPlan(b["offsets"], 5, tuning=tuning, degree=b["degree"])
    res = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, accum=accum, plan=plan,
                        basis="chebyshev")
    assert L.status_names(res["status"][5:6]) == ["invalid_arg"]
    good = [s for s in range(300) if s != 5]
    assert _check_cheb(L, b, res, accum, x.double().cpu().numpy(), y.double().cpu().numpy(), good) > 250
    # a monomial fit of the same batch gives the same polynomials
    mono = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, accum=accum, plan=plan)
    ok = (res["status"] == 0) & (mono["status"] == 0)
    assert int(ok.sum()) > 250


@pytest.mark.parametrize("dtype,accum", [(torch.float32, "comp"), (torch.bfloat16, "comp"),
                                         (torch.float32, "f64")])
def test_chebyshev_basis_high_degrees(L, dtype, accum):
    """Degrees 1..8 in one batch (the m_max = 8 kernel), in block and warp tasks."""
    # intervals wide enough for BF16 abscissae to stay distinct at degree 8
    b = synth.ragged_batch(num_series=120, lmin=64, lmax=30000, mmin=1, mmax=8, seed=46,
                           a_range=(-5.0, 5.0), w_range=(1.0, 8.0))
    x = torch.from_numpy(b["x"]).to(dtype).cuda()
    y = torch.from_numpy(b["y"]).to(dtype).cuda()
    plan = L.BatchPlan(b["offsets"], 8, tuning={"warp_max_len": 2048, "chunk_len": 8192}, degree=b["degree"])
    assert len(plan.block_tasks_host) > 0 and len(plan.warp_tasks_host) > 0
    res = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=8, accum=accum, plan=plan,
                        basis="chebyshev")
    assert _check_cheb(L, b, res, accum, x.double().cpu().numpy(), y.double().cpu().numpy()) > 100
    assert {int(m) for m in b["degree"]} == set(range(1, 9))


def test_chebyshev_basis_limits(L):
    b = synth.ragged_batch(num_series=20, lmin=16, lmax=3000, seed=45)
    x = torch.from_numpy(b["x"]).cuda()
    y = torch.from_numpy(b["y"]).cuda()
    with pytest.raises(L.LsefitError):  # no naive FP32 kernel in the Chebyshev basis
        L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, accum="naive", basis="chebyshev")
    res = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, accum="comp", basis="chebyshev")
    with pytest.raises(L.LsefitError):  # the adjoint differentiates the monomial normal equations
        L.backward(x, y, b["offsets"], b["degree"], res, torch.ones_like(res["X"]))
