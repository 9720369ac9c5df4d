"""Precision stress: 2^24 points, x on [0, 1000], degrees 1..8, FP32 and BF16 storage,
naive / compensated / FP64 accumulation, unscaled and mapped to [-1, 1].

Every result is compared with the oracle's FP64 fit of the same stored values in the
same basis, and the error of each coefficient is recorded with cond(A).  Forward gates
(relative 2-norm error of Xt):
  * FP64 accumulation: 1e-6 where cond(A) 2^-53 4m stays at or below 1e-3 (that is,
    everywhere but the unscaled fits of degree >= 2, which are reported);
  * compensated FP32 on the mapped interval: 1e-5 at every degree for FP32 storage
    (measured at most 3.1e-7, at m = 8) and for BF16 storage up to m = 6 (measured at
    most 8.8e-7); BF16 at m = 7, 8 is reported (1.3e-5 and 4.6e-5 measured: the
    rounding errors of repeated BF16 abscissae do not average out);
  * naive FP32 and the unscaled FP32 fits are reported.
Every ok result whose oracle status is ok also passes the backward-error gate of its
accumulation (tests/gates.py), which holds whatever cond(A) is.  Statuses of gated,
well-determined systems must match the oracle's; unscaled FP32 power sums of x ~ 1000
overflow at high degree (status `nonfinite`; FP64 does not overflow).

With LSEFIT_PRECISION_REPORT=<path> the table is also written there as markdown.
"""
import os

import numpy as np
import pytest

import gates
import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1 << 24
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def L():
    import paper_1512_08017_gb300 as lib
    return lib


def _hankel(S, m):
    return np.array([[S[j + k] for k in range(m + 1)] for j in range(m + 1)])


def _errs(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    norm = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
    per = float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)))
    return norm, per


def test_precision_grid(L):
    rows = []
    failures = []
    for m in range(1, 9):
        d = synth.precision(n=N, m=m)
        lo, hi = d["interval"]
        for storage in ("f32", "bf16"):
            if storage == "f32":
                xs, ys = d["x"].astype(np.float64), d["y"].astype(np.float64)
                x = torch.from_numpy(d["x"]).cuda()
                y = torch.from_numpy(d["y"]).cuda()
            else:
                xs = synth.from_bf16_bits(d["x_bf16"]).astype(np.float64)
                ys = synth.from_bf16_bits(d["y_bf16"]).astype(np.float64)
                x = torch.from_numpy(d["x_bf16"].view(np.int16)).view(torch.bfloat16).cuda()
                y = torch.from_numpy(d["y_bf16"].view(np.int16)).view(torch.bfloat16).cuda()
            refs = {}
            for mapped in (False, True):
                for accum in ("naive", "comp", "f64"):
                    fp32 = accum != "f64"
                    key = (mapped, fp32)
                    if key not in refs:
                        if mapped:
                            refs[key] = oracle.fit_interval(xs, ys, m, lo, hi, fp32=fp32)
                        else:
                            refs[key] = oracle.fit(xs, ys, m, eps=oracle.EPS32 if fp32 else oracle.EPS64)
                    ref = refs[key]
                    out = L.fit(x, y, m, accum=accum, interval=(lo, hi) if mapped else None)
                    st = L.status_names(out["status"])[0]
                    cond = float(np.linalg.cond(_hankel(ref["S"], m))) if ref["S"] is not None else float("nan")
                    row = {"m": m, "storage": storage, "map": "mapped" if mapped else "unscaled", "accum": accum,
                           "status": st, "oracle": ref["status"], "cond": cond}
                    if st == "ok" and ref["status"] == "ok":
                        row["xt_norm"], row["xt_max"] = _errs(out["Xt"].cpu().numpy(), ref["Xt"])
                        row["x_norm"], row["x_max"] = _errs(out["X"].cpu().numpy(), ref["X"])
                        row["eta"] = gates.backward_error(_hankel(ref["S"], m), ref["T"], out["Xt"].cpu().numpy())
                        if row["eta"] > gates.backward_gate(accum, N):
                            failures.append(("backward", row))
                    rows.append(row)
                    eps = 2.0 ** -53 if accum == "f64" else EPS32
                    if accum == "f64":
                        tol = gates.forward_gate("f64", m, cond)
                    elif accum == "comp" and mapped:
                        tol = 1e-5 if (storage == "f32" or m <= 6) else None
                    else:
                        tol = None  # reported only
                    # a gated case whose system is well determined (cond(A) eps < 1e-2) must
                    # reach the oracle's status; elsewhere the singular/non-singular call
                    # sits near the threshold and FP32 overflows unscaled high powers
                    determined = tol is not None and cond * eps < 1e-2
                    if st != ref["status"]:
                        if determined:
                            failures.append(("status", row))
                        continue
                    if st != "ok" or tol is None:
                        continue
                    row["tol"] = tol
                    if row["xt_norm"] > tol:
                        failures.append(("error", row))
    path = os.environ.get("LSEFIT_PRECISION_REPORT")
    if path:
        with open(path, "w") as f:
            f.write("| m | storage | x | accum | status (GPU / oracle) | cond(A) | Xt rel. error (norm / worst coef.) "
                    "| X rel. error (norm / worst coef.) | gate | backward error (gate) |\n"
                    "|---|---|---|---|---|---|---|---|---|---|\n")
            for r in rows:
                e1 = f"{r['xt_norm']:.2e} / {r['xt_max']:.2e}" if "xt_norm" in r else "—"
                e2 = f"{r['x_norm']:.2e} / {r['x_max']:.2e}" if "x_norm" in r else "—"
                gate = f"{r['tol']:.1e}" if r.get("tol") else "reported"
                eta = f"{r['eta']:.1e} ({gates.backward_gate(r['accum'], N):.1e})" if "eta" in r else "—"
                f.write(f"| {r['m']} | {r['storage']} | {r['map']} | {r['accum']} | {r['status']} / {r['oracle']} "
                        f"| {r['cond']:.2e} | {e1} | {e2} | {gate} | {eta} |\n")
    assert not failures, failures[:5]
