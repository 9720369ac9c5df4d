"""The C boundary used from C: tests/c_client/fit_client.c (CUDA runtime and
liblsefit.so only, no Python on the data path) fits one series and a small
ragged batch; its printed coefficients are checked against the oracle."""
import glob
import os
import shutil
import subprocess

import numpy as np
import pytest

import gates
import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_lib_dir():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for cand in [os.path.join(home, "lib64")] + sorted(glob.glob(os.path.join(home, "targets", "*", "lib"))):
        if os.path.exists(os.path.join(cand, "libcudart.so")):
            return home, cand
    pytest.skip("libcudart.so not found")


def test_c_client(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1512_08017_gb300 import _build
    _build.build()
    home, cudalib = _cuda_lib_dir()
    exe = str(tmp_path / "fit_client")
    cmd = ["gcc", "-O2", "-std=c99", os.path.join(ROOT, "tests", "c_client", "fit_client.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(home, "include"),
           "-L", _build.LIB_DIR, "-llsefit", "-L", cudalib, "-lcudart",
           f"-Wl,-rpath,{_build.LIB_DIR}", f"-Wl,-rpath,{cudalib}", "-o", exe]
    subprocess.run(cmd, check=True)

    d = synth.single_large(n=50_000, m=3, seed=123)
    x, y = d["x"], d["y"]
    rng = np.random.default_rng(124)
    cuts = np.sort(rng.choice(np.arange(1, x.size), 19, replace=False))
    offsets = np.concatenate([[0], cuts, [x.size]]).astype(np.int64)
    degree = rng.integers(1, 6, offsets.size - 1).astype(np.int32)
    inp = tmp_path / "input.txt"
    with open(inp, "w") as f:
        f.write(f"{x.size}\n")
        f.writelines(f"{a!r} {b!r}\n" for a, b in zip(x.tolist(), y.tolist()))
        f.write(f"{offsets.size - 1}\n" + " ".join(map(str, offsets)) + "\n" + " ".join(map(str, degree)) + "\n")
    out = subprocess.run([exe, str(inp)], check=True, capture_output=True, text=True).stdout.splitlines()

    xs, ys = x.astype(np.float64), y.astype(np.float64)
    single = [l.split() for l in out if l.startswith("single")]
    assert len(single) == 3
    for row in single:
        m, st = int(row[1]), int(row[2])
        got = np.array([float(v) for v in row[3:]])[: m + 1]
        ref = oracle.fit_interval(xs, ys, m, -1.0, 1.0, fp32=True)
        assert st == 0 and ref["status"] == "ok"
        assert np.linalg.norm(got - ref["X"]) <= 1e-5 * np.linalg.norm(ref["X"])
    batch = [l.split() for l in out if l.startswith("batch")]
    assert len(batch) == offsets.size - 1
    for row in batch:
        s, st = int(row[1]), int(row[2])
        lo, hi = offsets[s], offsets[s + 1]
        m = int(degree[s])
        ref = oracle.fit(xs[lo:hi], ys[lo:hi], m, eps=oracle.EPS32)
        if ref["status"] != "ok":
            continue
        assert st == 0
        got = np.array([float(v) for v in row[3:]])
        # no interval: X = Xt; forward gate where it applies, backward gate always
        gates.check_coefficients(got, ref["X"], gates.hankel(ref["S"], m), ref["T"], "comp", m)
