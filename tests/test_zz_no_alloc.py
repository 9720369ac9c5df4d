"""The allocation-free entry point gives the same fit as lsefit_fit.

lsefit_fit_noalloc serves callers that cannot allocate device memory when
they fit (a service with a fixed device-memory budget that forbids
allocation after start-up, or a plugin host that passes only input and
output buffers).  Its scratch is a static array inside the library, shared
by every call, so the test makes two calls in a row on different data and
compares each with lsefit_fit (which uses a caller workspace) through the
C ABI, within the tolerance the GPU-to-GPU comparisons of this suite use
(relative 1e-12), and with the oracle within the compensated-FP32 tolerance
(1e-5, degree <= 3 on [-1, 1]).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _outputs(k, m, dev):
    return {"X": torch.full((k, m + 1), float("nan"), dtype=torch.float64, device=dev),
            "Xt": torch.full((k, m + 1), float("nan"), dtype=torch.float64, device=dev),
            "sums": torch.full((3 * m + 2,), float("nan"), dtype=torch.float64, device=dev),
            "map": torch.full((2,), float("nan"), dtype=torch.float64, device=dev),
            "status": torch.full((k,), -1, dtype=torch.int32, device=dev)}


def test_noalloc_matches_lsefit_fit_twice():
    from paper_1512_08017_gb300 import lsefit as B

    dev = torch.device("cuda", torch.cuda.current_device())
    m, m_lo = 3, 1
    k = m - m_lo + 1
    assert B.lib.lsefit_fit_noalloc_scratch_bytes() >= B.lib.lsefit_powersums_workspace_size(8)
    iv = torch.tensor([-1.0, 1.0], dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for call, (n, seed) in enumerate([((1 << 20) + 5, 71), ((1 << 18) + 3, 72)]):
        d = synth.single_large(n=n, m=m, seed=seed)
        x = torch.from_numpy(d["x"]).to(dev)
        y = torch.from_numpy(d["y"]).to(dev)
        # the existing entry point, with its own zero-filled workspace
        ws = torch.zeros(B.lib.lsefit_powersums_workspace_size(m), dtype=torch.uint8, device=dev)
        ref = _outputs(k, m, dev)
        rc = B.lib.lsefit_fit(B._ptr(x), B._ptr(y), n, B.F32, m, m_lo, B.ACCUM["comp"], B._ptr(iv),
                              B._ptr(ref["X"]), B._ptr(ref["Xt"]), B._ptr(ref["sums"]), B._ptr(ref["map"]),
                              B._ptr(ref["status"]), B._ptr(ws), ws.numel(), ctypes.c_void_p(stream.cuda_stream))
        assert rc == B.OK
        # the allocation-free entry point
        out = _outputs(k, m, dev)
        rc = B.lib.lsefit_fit_noalloc(B._ptr(x), B._ptr(y), n, B.F32, m, m_lo, B.ACCUM["comp"], B._ptr(iv),
                                      B._ptr(out["X"]), B._ptr(out["Xt"]), B._ptr(out["sums"]),
                                      B._ptr(out["map"]), B._ptr(out["status"]),
                                      ctypes.c_void_p(stream.cuda_stream))
        assert rc == B.OK, B.status_string(rc)
        torch.cuda.synchronize()
        assert out["status"].tolist() == [B.OK] * k, call
        for key in ("X", "Xt", "sums", "map"):
            assert _rel(out[key].cpu().numpy(), ref[key].cpu().numpy()) <= 1e-12, (call, key)
        for r, deg in enumerate(range(m_lo, m + 1)):
            o = oracle.fit_interval(d["x"], d["y"], deg, -1.0, 1.0, fp32=True)
            assert _rel(out["Xt"][r, : deg + 1].cpu().numpy(), o["Xt"]) <= 1e-5, (call, deg)


def _fit_both(B, x, y, n, m, m_lo, iv, dev, stream):
    """lsefit_fit (own zero-filled workspace) and lsefit_fit_noalloc on the same input."""
    k = m - m_lo + 1
    ws = torch.zeros(B.lib.lsefit_powersums_workspace_size(m), dtype=torch.uint8, device=dev)
    ref = _outputs(k, m, dev)
    rc = B.lib.lsefit_fit(B._ptr(x), B._ptr(y), n, B.F32, m, m_lo, B.ACCUM["comp"], B._ptr(iv),
                          B._ptr(ref["X"]), B._ptr(ref["Xt"]), B._ptr(ref["sums"]), B._ptr(ref["map"]),
                          B._ptr(ref["status"]), B._ptr(ws), ws.numel(), ctypes.c_void_p(stream.cuda_stream))
    assert rc == B.OK
    out = _outputs(k, m, dev)
    rc = B.lib.lsefit_fit_noalloc(B._ptr(x), B._ptr(y), n, B.F32, m, m_lo, B.ACCUM["comp"], B._ptr(iv),
                                  B._ptr(out["X"]), B._ptr(out["Xt"]), B._ptr(out["sums"]), B._ptr(out["map"]),
                                  B._ptr(out["status"]), ctypes.c_void_p(stream.cuda_stream))
    assert rc == B.OK, B.status_string(rc)
    torch.cuda.synchronize()
    return ref, out


def test_noalloc_reuse_at_other_shapes_and_after_rejected_calls():
    """The shared array reused at another degree and grid (m = 8 after m = 3,
    then m = 1 on fewer points), and after calls the entry point rejects
    (bad degree, missing status): each result equals lsefit_fit's."""
    from paper_1512_08017_gb300 import lsefit as B

    dev = torch.device("cuda", torch.cuda.current_device())
    iv = torch.tensor([-1.0, 1.0], dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    cases = [((1 << 19) + 7, 8, 6, 81), ((1 << 12) + 1, 1, 1, 82), ((1 << 20) + 3, 3, 1, 83)]
    for i, (n, m, m_lo, seed) in enumerate(cases):
        d = synth.single_large(n=n, m=min(m, 4), seed=seed)
        x = torch.from_numpy(d["x"]).to(dev)
        y = torch.from_numpy(d["y"]).to(dev)
        if i == 1:
            # rejected before any launch: the next call must be unaffected
            bad = _outputs(1, 1, dev)
            assert B.lib.lsefit_fit_noalloc(B._ptr(x), B._ptr(y), n, B.F32, 9, 1, B.ACCUM["comp"], B._ptr(iv),
                                            B._ptr(bad["X"]), None, None, None, B._ptr(bad["status"]),
                                            ctypes.c_void_p(stream.cuda_stream)) == B.ERR_INVALID_ARG
            assert B.lib.lsefit_fit_noalloc(B._ptr(x), B._ptr(y), n, B.F32, 1, 1, B.ACCUM["comp"], B._ptr(iv),
                                            B._ptr(bad["X"]), None, None, None, None,
                                            ctypes.c_void_p(stream.cuda_stream)) == B.ERR_INVALID_ARG
        ref, out = _fit_both(B, x, y, n, m, m_lo, iv, dev, stream)
        k = m - m_lo + 1
        assert out["status"].tolist() == ref["status"].tolist() == [B.OK] * k, (i, m)
        for key in ("X", "Xt", "sums", "map"):
            assert _rel(out[key].cpu().numpy(), ref[key].cpu().numpy()) <= 1e-12, (i, key)
