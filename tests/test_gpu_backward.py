"""Parity of the CUDA adjoint (lsefit_backward) with the oracle's adjoint and with
FP64 central finite differences of the oracle's fit.

Tolerance (not fixed by the paper): relative 2-norm error <= 1e-4 per series
for FP32 data (the per-point values are formed in FP32: t, the Horner sums
and the residual y - f(t) each carry a few 2^-24 relative errors, and the
residual loses up to |y| / |r| of that to cancellation), 1e-8 for FP64 data.
Series of the ragged batch whose normal matrix makes that bound exceed 1e-3
(cond(A) 2^-24 8m) have their gradients reported, not gated; they are held
instead to the identity V^T dy = M^T gX (dy_i = lambda(t_i) and A lambda = M^T gX),
whose error does not grow with cond(A).
The loss is L = sum_j w_j X_j^2 with w ~ N(0, 1) per series and
coefficient, so gX = 2 w X.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_1512_08017_gb300 as lib
    return lib


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _run(L, xs, ys, offsets, degree, interval, m_max, w, dtype=torch.float32, accum="comp", tuning=None):
    dev = torch.device("cuda")
    x = torch.from_numpy(xs).to(dev).to(dtype)
    y = torch.from_numpy(ys).to(dev).to(dtype)
    plan = L.BatchPlan(offsets, m_max, tuning=tuning)
    fwd = L.fit_batched(x, y, offsets, degree, interval, m_max=m_max, accum=accum, plan=plan)
    gX = 2.0 * torch.from_numpy(w).cuda() * fwd["X"]
    dx, dy, st = L.backward(x, y, offsets, degree, fwd, gX, interval_given=interval is not None, accum=accum)
    torch.cuda.synchronize()
    return fwd, gX, dx.double().cpu().numpy(), dy.double().cpu().numpy(), st.cpu().numpy()


def _oracle_grads(xs, ys, lo, hi, m, interval, w_row, fp32_map=True):
    if interval is not None:
        r = oracle.fit_interval(xs[lo:hi], ys[lo:hi], m, *interval, fp32=fp32_map)
        cs = (r["c"], r["s"])
    else:
        r = oracle.fit(xs[lo:hi], ys[lo:hi], m)
        cs = None
    gX = 2.0 * w_row[: m + 1] * r["X"]
    st, dx, dy = oracle.backward(xs[lo:hi], ys[lo:hi], m, cs, r["S"], r["Xt"], gX)
    return st, dx, dy, r, cs


def _identity_error(x, dy, r, w_row, m):
    """Largest relative defect of V^T dy = M^T gX over k = 0..m, where V holds the
    powers of the mapped abscissae and M is the un-map (columns: oracle.unmap of
    unit vectors).  Each defect is relative to sum_i |t_i|^k |lambda|(|t_i|) + |g_k|,
    lambda = A^-1 M^T gX from the oracle's sums, the size of the terms whose
    roundings it collects."""
    t = r["s"] * (x - r["c"])
    M = np.stack([oracle.unmap(np.eye(m + 1)[k], r["c"], r["s"]) for k in range(m + 1)], axis=1)
    g = M.T @ (2.0 * w_row[: m + 1] * r["X"])
    A = np.array([[r["S"][j + k] for k in range(m + 1)] for j in range(m + 1)])
    lam = np.linalg.solve(A, g)
    at = np.abs(t)
    lam_abs = sum(abs(lam[j]) * at ** j for j in range(m + 1))
    worst = 0.0
    for k in range(m + 1):
        got = float(np.sum(t ** k * dy))
        scale = float(np.sum(at ** k * lam_abs)) + abs(g[k])
        worst = max(worst, abs(got - g[k]) / scale)
    return worst


@pytest.mark.parametrize("with_interval", [True, False])
def test_uniform_batch_against_oracle_adjoint(L, with_interval):
    d = synth.diff_batch(num_series=64, n=512, seed=51)
    S, n = d["x"].shape
    offsets = np.arange(S + 1, dtype=np.int64) * n
    degree = np.full(S, 3, dtype=np.int32)
    interval = np.tile([-1.0, 1.0], (S, 1)) if with_interval else None
    xs, ys = d["x"].reshape(-1), d["y"].reshape(-1)
    fwd, gX, dx, dy, st = _run(L, xs, ys, offsets, degree, interval, 3, d["w"])
    assert np.all(st == 0)
    x64, y64 = xs.astype(np.float64), ys.astype(np.float64)
    for s in range(S):
        lo, hi = s * n, (s + 1) * n
        ost, odx, ody, _, _ = _oracle_grads(x64, y64, lo, hi, 3, interval[s] if with_interval else None,
                                            d["w"][s])
        assert ost == "ok"
        assert _rel(dy[lo:hi], ody) <= 1e-4, s
        assert _rel(dx[lo:hi], odx) <= 1e-4, s


def test_ragged_mixed_degrees_against_oracle_adjoint(L):
    b = synth.ragged_batch(num_series=200, lmin=8, lmax=30000, seed=52)
    w = np.random.default_rng(52).normal(size=(200, 6))
    for tuning in (None, {"warp_max_len": 256, "chunk_len": 2048}):
        fwd, gX, dx, dy, st = _run(L, b["x"], b["y"], b["offsets"], b["degree"], b["interval"], 5, w,
                                   tuning=tuning)
        x64, y64 = b["x"].astype(np.float64), b["y"].astype(np.float64)
        fst = fwd["status"].cpu().numpy()
        for s in range(200):
            lo, hi = int(b["offsets"][s]), int(b["offsets"][s + 1])
            m = int(b["degree"][s])
            ost, odx, ody, r, _ = _oracle_grads(x64, y64, lo, hi, m, b["interval"][s], w[s])
            if r["status"] != "ok":
                assert fst[s] != 0 and st[s] != 0
                assert np.all(dx[lo:hi] == 0) and np.all(dy[lo:hi] == 0)
                continue
            assert st[s] == 0
            A = np.array([[r["S"][j + k] for k in range(m + 1)] for j in range(m + 1)])
            tol = max(1e-4, np.linalg.cond(A) * 2.0 ** -24 * 8 * m)
            if tol <= 1e-3:
                assert _rel(dy[lo:hi], ody) <= tol, (s, m, hi - lo)
                assert _rel(dx[lo:hi], odx) <= tol, (s, m, hi - lo)
            assert _identity_error(x64[lo:hi], dy[lo:hi], r, w[s], m) <= 1e-4, (s, m, hi - lo)


def test_central_differences_subset(L):
    # the differentiable-fit workload shape on a 64-series subset: FP64 central
    # differences (h = 1e-6) of the oracle's loss, per point and along random directions
    d = synth.diff_batch(num_series=64, n=4096, seed=53)
    S, n = d["x"].shape
    offsets = np.arange(S + 1, dtype=np.int64) * n
    degree = np.full(S, 3, dtype=np.int32)
    interval = np.tile([-1.0, 1.0], (S, 1))
    xs, ys = d["x"].reshape(-1), d["y"].reshape(-1)
    fwd, gX, dx, dy, st = _run(L, xs, ys, offsets, degree, interval, 3, d["w"])
    x64, y64 = xs.astype(np.float64), ys.astype(np.float64)
    h = 1e-6
    rng = np.random.default_rng(54)
    _, c, sc = oracle.map_constants(-1.0, 1.0, True)

    def loss(xv, yv, s):
        return float(np.sum(d["w"][s] * oracle.fit(xv, yv, 3, (c, sc))["X"] ** 2))

    for s in range(S):
        lo, hi = s * n, (s + 1) * n
        xv, yv = x64[lo:hi].copy(), y64[lo:hi].copy()
        gscale_x = np.max(np.abs(dx[lo:hi]))
        gscale_y = np.max(np.abs(dy[lo:hi]))
        for i in rng.choice(n, 3, replace=False):
            e = np.zeros(n)
            e[i] = h
            fdy = (loss(xv, yv + e, s) - loss(xv, yv - e, s)) / (2 * h)
            fdx = (loss(xv + e, yv, s) - loss(xv - e, yv, s)) / (2 * h)
            assert abs(fdy - dy[lo + i]) <= 1e-4 * gscale_y + 1e-9, (s, i)
            assert abs(fdx - dx[lo + i]) <= 1e-4 * gscale_x + 1e-9, (s, i)
        v = rng.normal(size=n)
        v /= np.linalg.norm(v)
        fd = (loss(xv + h * v, yv, s) - loss(xv - h * v, yv, s)) / (2 * h)
        assert abs(fd - v @ dx[lo:hi]) <= 1e-4 * np.linalg.norm(dx[lo:hi]) + 1e-9
        fd = (loss(xv, yv + h * v, s) - loss(xv, yv - h * v, s)) / (2 * h)
        assert abs(fd - v @ dy[lo:hi]) <= 1e-4 * np.linalg.norm(dy[lo:hi]) + 1e-9


def test_autograd_function(L):
    d = synth.diff_batch(num_series=32, n=1000, seed=55)
    S, n = d["x"].shape
    offsets = np.arange(S + 1, dtype=np.int64) * n
    degree = np.full(S, 3, dtype=np.int32)
    interval = np.tile([-1.0, 1.0], (S, 1))
    x = torch.from_numpy(d["x"].reshape(-1)).cuda().requires_grad_(True)
    y = torch.from_numpy(d["y"].reshape(-1)).cuda().requires_grad_(True)
    X, status = L.fit_differentiable(x, y, offsets, degree, interval, m_max=3)
    w = torch.from_numpy(d["w"]).cuda()
    (w * X ** 2).sum().backward()
    assert torch.all(status == 0)
    _, _, dx, dy, _ = _run(L, d["x"].reshape(-1), d["y"].reshape(-1), offsets, degree, interval, 3, d["w"])
    np.testing.assert_allclose(x.grad.double().cpu().numpy(), dx, rtol=0, atol=1e-6 * np.max(np.abs(dx)))
    np.testing.assert_allclose(y.grad.double().cpu().numpy(), dy, rtol=0, atol=1e-6 * np.max(np.abs(dy)))


def test_fp64_storage(L):
    b = synth.ragged_batch(num_series=60, lmin=16, lmax=5000, seed=56, a_range=(-3.0, 3.0),
                           w_range=(1.0, 5.0))
    xs, ys = b["x"].astype(np.float64), b["y"].astype(np.float64)
    w = np.random.default_rng(56).normal(size=(60, 6))
    fwd, gX, dx, dy, st = _run(L, xs, ys, b["offsets"], b["degree"], b["interval"], 5, w,
                               dtype=torch.float64, accum="f64")
    for s in range(60):
        lo, hi = int(b["offsets"][s]), int(b["offsets"][s + 1])
        m = int(b["degree"][s])
        ost, odx, ody, r, _ = _oracle_grads(xs, ys, lo, hi, m, b["interval"][s], w[s], fp32_map=False)
        if r["status"] != "ok":
            continue
        assert _rel(dy[lo:hi], ody) <= 1e-8, s
        assert _rel(dx[lo:hi], odx) <= 1e-8, s
