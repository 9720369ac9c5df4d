"""Host logic of bench.py (no GPU): the traffic record tied to the CUDA sources
it was captured on, the peaks file and its fallback, the host description, and
the defaults the timing contract asks for."""
import json
import os
import shutil

import bench


def _fake_root(tmp_path, with_csrc=True):
    root = tmp_path / "root"
    (root / "profiles").mkdir(parents=True)
    if with_csrc:
        shutil.copytree(os.path.join(bench.ROOT, "paper_1512_08017_gb300", "csrc"),
                        root / "paper_1512_08017_gb300" / "csrc")
    return root


def test_source_digest_follows_the_kernel_sources(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    (root / "include").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "include", "lsefit.h"), root / "include" / "lsefit.h")
    keys = ("powersums_f32_comp_m3", "residuals_f32", "batched_f32_comp", "general_weighted", "diff_fwd_bwd")
    real = {k: bench.source_digest(k) for k in keys + (None,)}
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert {k: bench.source_digest(k) for k in keys + (None,)} == real
    # a kernel's own file changes its digest only
    f = root / "paper_1512_08017_gb300" / "csrc" / "lsefit_residuals.cu"
    f.write_text(f.read_text() + "\n// edited\n")
    assert bench.source_digest("residuals_f32") != real["residuals_f32"]
    assert bench.source_digest(None) != real[None]
    for k in ("powersums_f32_comp_m3", "batched_f32_comp", "general_weighted", "diff_fwd_bwd"):
        assert bench.source_digest(k) == real[k], k
    # a shared header changes every digest
    g = root / "paper_1512_08017_gb300" / "csrc" / "lsefit_device.cuh"
    g.write_text(g.read_text() + "\n// edited\n")
    for k in keys:
        assert bench.source_digest(k) != real[k], k


def test_recorded_traffic_only_for_the_current_sources(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    (root / "include").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "include", "lsefit.h"), root / "include" / "lsefit.h")
    monkeypatch.setattr(bench, "ROOT", str(root))
    dig = bench.source_digest("k_now")
    rec = {"k_now": {"source_digest": dig, "dram_bytes_per_launch": 123.0},
           "k_old": {"source_digest": "0" * 16, "dram_bytes_per_launch": 456.0}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("k_now") == 123.0
    assert bench.recorded_traffic("k_old") is None      # captured on other sources: null
    assert bench.recorded_traffic("missing") is None
    (root / "profiles" / "traffic.json").write_text("not json")
    assert bench.recorded_traffic("k_now") is None


def test_committed_traffic_records_are_well_formed():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for key in ("powersums_f32_comp_m3", "batched_f32_comp", "residuals_f32", "diff_fwd_bwd",
                "general_weighted", "general_chebyshev"):
        v = rec[key]
        assert len(v["source_digest"]) == 16 and v["dram_bytes_per_launch"] > 0
        assert abs(v["dram_bytes_per_launch"] - v["captured_bytes"] * v["scale"]) <= 1e-6 * v["captured_bytes"] * v["scale"]
        assert v["kernels"] and v["note"]


def test_measured_peaks_and_fallback(tmp_path, monkeypatch):
    root = _fake_root(tmp_path, with_csrc=False)
    monkeypatch.setattr(bench, "ROOT", str(root))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0
    (root / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.0, "bf16_tflops": 2000.0}))
    peaks, kind = bench.measured_peaks()
    assert kind == "measured" and peaks["hbm_gbs"] == 7000.0


def test_host_info():
    h = bench.host_info()
    assert h["nproc"] >= 1 and h["machine"]


def test_contract_defaults():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.impl == "lsefit" and a.workload == "single_large"
    assert a.warmup >= 3 and a.steps >= 1
    assert a.n == 1 << 28


def test_error_helpers():
    """The coefficient-error helpers of the bench line: the backward error of an
    exact solution of the normal equations is at rounding level, that of a
    perturbed one is not; rel_err is the normwise relative error."""
    import numpy as np
    S = np.array([4.0, 2.0, 3.0, 2.5, 2.8])  # S_0..S_4 of a degree-2 system
    A = np.array([[S[j + k] for k in range(3)] for j in range(3)])
    X = np.array([0.5, -1.0, 2.0])
    T = A @ X
    assert bench.backward_err(S, T, 2, X) < 1e-15
    assert bench.backward_err(S, T, 2, X * (1 + 1e-6)) > 1e-8
    assert abs(bench.rel_err([1.0, 2.0], [1.0, 2.0])) == 0.0
    assert abs(bench.rel_err([1.0, 2.1], [1.0, 2.0]) - 0.1 / np.sqrt(5.0)) < 1e-15


def test_host_placement_helpers():
    import numpy as np
    a = np.ones(1 << 16)
    node = bench.page_node(a.ctypes.data)
    assert node is None or node >= 0
    nodes = bench.numa_nodes_with_cpus()
    assert isinstance(nodes, dict)
    for k, v in nodes.items():
        assert k >= 0 and isinstance(v, str)


def test_general_coefficient_record():
    """coef_err_general: zero error for the oracle's own solution, a planted
    error shows in both coefficient sets and in the backward error, and a status
    other than ok reports no error figures."""
    import numpy as np
    import oracle
    import synth
    d = synth.small_series(5000, seed=3, lo=-1.0, hi=1.0, m=4, dtype=np.float64)
    ref = oracle.fit_general_interval(d["x"].astype(np.float32), d["y"].astype(np.float32), 4, -1.0, 1.0,
                                      fp32=True, basis="chebyshev")
    out = {"Xb": np.tile(np.append(ref["Xb"], 0.0), (4, 1)), "X": np.tile(np.append(ref["X"], 0.0), (4, 1))}
    rec = bench.coef_err_general(out, ref, 4, "comp", 5000, "ok")
    assert rec["rel_Xb"] == 0.0 and rec["rel_X"] == 0.0 and rec["backward"] < 1e-15
    assert rec["forward_gate"] == 1e-5 and rec["backward_gate"] == 1e-5
    out["Xb"][3, 2] *= 1.1
    out["X"][3, 2] *= 1.1
    bad = bench.coef_err_general(out, ref, 4, "comp", 5000, "ok")
    assert bad["rel_Xb"] > 1e-5 and bad["rel_X"] > 1e-5 and bad["backward"] > 1e-6
    assert bench.coef_err_general(out, ref, 4, "f64", 5000, "singular") == {
        "degree": 4, "status": "singular", "oracle_status": "ok"}


def test_timed_region_is_one_event_pair(monkeypatch):
    """The K timed steps run back to back between one pair of events on the
    launching stream (an event pair around every step separates consecutive graph
    launches); the result is the pair's elapsed time."""
    import torch
    log = []

    class FakeEvent:
        def __init__(self, enable_timing=False):
            assert enable_timing
            self.at = None

        def record(self, stream=None):
            log.append(("record", stream))
            self.at = len(log)

        def elapsed_time(self, other):
            return float(other.at - self.at)

    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: log.append(("sync",)))
    stream = object()
    total = bench._event_steps(lambda: log.append(("step",)), 7, stream)
    assert log == [("record", stream)] + [("step",)] * 7 + [("record", stream), ("sync",)]
    assert total == 8.0
