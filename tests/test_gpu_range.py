"""The interval prepass (lsefit_range) returns each series' exact [min x, max x]."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_1512_08017_gb300 as lib
    return lib


def _expected(x64, offsets):
    out = np.full((len(offsets) - 1, 2), np.nan)
    for s in range(len(offsets) - 1):
        seg = x64[offsets[s]: offsets[s + 1]]
        seg = seg[~np.isnan(seg)]
        if seg.size:
            out[s] = (seg.min(), seg.max())
    return out


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
@pytest.mark.parametrize("tuning", [None, {"warp_max_len": 64, "chunk_len": 1024}])
def test_range_exact(L, dtype, tuning):
    lengths = np.array([0, 1, 2, 7, 100, 5000, 70000, 3, 0, 40000])
    b = synth.ragged_batch(lengths=lengths, seed=81)
    off = b["offsets"]
    b["x"][off[4] + 10] = np.nan          # NaN points are ignored
    b["x"][off[7]: off[8]] = np.nan       # a series of NaN only
    x = torch.from_numpy(b["x"]).to(dtype).cuda()
    plan = L.BatchPlan(off, 5, tuning=tuning)
    got = L.range_batched(x, off, plan=plan).cpu().numpy()
    exp = _expected(x.double().cpu().numpy(), off)
    assert np.array_equal(np.isnan(got), np.isnan(exp))
    ok = ~np.isnan(exp)
    assert np.array_equal(got[ok], exp[ok])
    # the workspace is left zeroed: a second call gives the same answer
    got2 = L.range_batched(x, off, plan=plan).cpu().numpy()
    assert np.array_equal(np.nan_to_num(got2), np.nan_to_num(got))


def test_range_then_fit_matches_given_interval(L):
    b = synth.ragged_batch(num_series=200, lmin=16, lmax=20000, seed=82)
    x = torch.from_numpy(b["x"]).cuda()
    y = torch.from_numpy(b["y"]).cuda()
    iv = L.range_batched(x, b["offsets"])
    exp = _expected(b["x"].astype(np.float64), b["offsets"])
    assert np.array_equal(iv.cpu().numpy(), exp)
    res = L.fit_batched(x, y, b["offsets"], b["degree"], iv, m_max=5, accum="comp")
    assert L.status_names(res["status"]).count("ok") == 200
