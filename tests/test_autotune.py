"""Host logic of the autotuner of the batched schedule (no GPU): the layout
signature, the cache and its key, the built-in candidates and the device
buffer sizes the C autotuner asks for, and its argument checks."""
import ctypes
import json

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def A():
    from paper_1512_08017_gb300 import _build
    _build.build()
    from paper_1512_08017_gb300 import autotune
    return autotune


def _offsets(lengths):
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def test_layout_signature_stable_and_separating(A):
    rng = np.random.default_rng(5)
    lens = synth.ragged_lengths(5000, 16, 65536, rng)
    sig = A.layout_signature(_offsets(lens))
    # a handful of series one point longer or shorter: the same layout
    near = lens.copy()
    near[rng.choice(lens.size, 20, replace=False)] += 1
    near[rng.choice(lens.size, 20, replace=False)] -= 1
    assert A.layout_signature(_offsets(near)) == sig
    # other series counts, other length distributions, other totals: different layouts
    assert A.layout_signature(_offsets(lens[:4000])) != sig
    assert A.layout_signature(_offsets(np.full(5000, int(lens.mean())))) != sig
    assert A.layout_signature(_offsets(lens * 4)) != sig
    assert A.layout_signature(_offsets(np.full(4096, 4096))) == A.layout_signature(_offsets(np.full(4096, 4096)))


def test_cache_key_holds_device_driver_and_layout(A):
    k = A.cache_key("GB300", 152, 13000, "torch.float32", "comp", 5, "S1:N2:H3")
    assert "GB300" in k and "|152|" in k and "drv13000" in k and "S1:N2:H3" in k and "m5" in k
    assert k != A.cache_key("GB300", 152, 13010, "torch.float32", "comp", 5, "S1:N2:H3")  # another driver
    assert k != A.cache_key("GB300", 152, 13000, "torch.float32", "comp", 5, "S1:N2:H3", basis="chebyshev")
    assert k != A.cache_key("GB300", 148, 13000, "torch.float32", "comp", 5, "S1:N2:H3")


def test_cache_round_trip_and_corrupt_file(A, tmp_path, monkeypatch):
    monkeypatch.setenv("LSEFIT_CACHE_DIR", str(tmp_path))
    assert A.load_cache() == {}
    entry = {"tuning": {"warp_max_len": 4096, "chunk_len": 65536, "schedule": 3}, "ms": 0.5, "candidates": []}
    A.store_cache({"k1": entry})
    assert A.load_cache() == {"k1": entry}
    # a corrupt file, a file of another shape and entries without a tuning are ignored
    path = tmp_path / "autotune.json"
    path.write_text("{not json")
    assert A.load_cache() == {}
    path.write_text(json.dumps([1, 2, 3]))
    assert A.load_cache() == {}
    path.write_text(json.dumps({"k1": entry, "k2": {"ms": 1.0}, "k3": "x"}))
    assert A.load_cache() == {"k1": entry}


def test_builtin_candidates_and_sizes(A):
    from paper_1512_08017_gb300 import lsefit as L
    cands = A.builtin_candidates()
    assert len(cands) == 7 and {c["schedule"] for c in cands} == {1, 2, 3}
    assert len(cands) <= 32
    b = synth.ragged_batch(num_series=3000, lmin=16, lmax=300000, seed=8, threads=1)
    off, deg = b["offsets"], b["degree"]
    n = len(cands)
    arr = (L.Tuning * n)(*[A._tuning_struct(c) for c in cands])
    ints, ws = ctypes.c_int64(0), ctypes.c_size_t(0)
    rc = L.lib.lsefit_plan_autotune_sizes(off.ctypes.data_as(ctypes.c_void_p), deg.ctypes.data_as(ctypes.c_void_p),
                                          off.size - 1, 5, arr, n, 152, ctypes.byref(ints), ctypes.byref(ws))
    assert rc == L.OK
    # the sizes cover every candidate's plan
    for c in cands:
        plan = L.Plan()
        rc = L.lib.lsefit_plan_build(off.ctypes.data_as(ctypes.c_void_p), deg.ctypes.data_as(ctypes.c_void_p),
                                     off.size - 1, 5, ctypes.byref(A._tuning_struct(c)), 152, ctypes.byref(plan),
                                     None, 0, None, 0)
        assert rc in (L.OK, L.ERR_WORKSPACE)
        assert 4 * (plan.n_block_tasks + plan.n_warp_tasks) <= ints.value
        assert L.lib.lsefit_batched_workspace_size(ctypes.byref(plan)) <= ws.value
    # NULL candidates = the built-in list
    ints2, ws2 = ctypes.c_int64(0), ctypes.c_size_t(0)
    assert L.lib.lsefit_plan_autotune_sizes(off.ctypes.data_as(ctypes.c_void_p), None, off.size - 1, 5, None, 0,
                                            152, ctypes.byref(ints2), ctypes.byref(ws2)) == L.OK
    assert ints2.value == ints.value and ws2.value == ws.value


def test_autotune_argument_errors_before_any_cuda_call(A):
    from paper_1512_08017_gb300 import lsefit as L
    off = np.array([0, 10, 30], dtype=np.int64)
    b = L.Batch(None, None, None, None, None, 2, 3, L.F32, 1, 0)
    best = L.Tuning()
    buf = (ctypes.c_int32 * 64)()
    offp = off.ctypes.data_as(ctypes.c_void_p)
    f = L.lib.lsefit_plan_autotune
    # no batch, no outputs, no repetitions, too many candidates
    assert f(None, offp, None, None, 0, 1, buf, 64, buf, 256, buf, buf, None, ctypes.byref(best), None) == L.ERR_INVALID_ARG
    assert f(ctypes.byref(b), offp, None, None, 0, 1, buf, 64, buf, 256, None, buf, None, ctypes.byref(best),
             None) == L.ERR_INVALID_ARG
    assert f(ctypes.byref(b), offp, None, None, 0, 0, buf, 64, buf, 256, buf, buf, None, ctypes.byref(best),
             None) == L.ERR_INVALID_ARG
    many = (L.Tuning * 33)()
    assert f(ctypes.byref(b), offp, None, many, 33, 1, buf, 64, buf, 256, buf, buf, None, ctypes.byref(best),
             None) == L.ERR_INVALID_ARG
    # task buffer not 16-byte aligned
    mis = ctypes.c_void_p(ctypes.addressof(buf) + 4)
    assert f(ctypes.byref(b), offp, None, None, 0, 1, mis, 60, buf, 256, buf, buf, None, ctypes.byref(best),
             None) == L.ERR_WORKSPACE
    assert L.lib.lsefit_driver_version() >= 0
