#!/usr/bin/env python
"""Throughput benchmark of the least-squares polynomial fit on one or more GPUs.

Default workload (one step = one whole fit): a single series of n = 2^28
FP32 points (2 GiB of x, y; larger than L2, so no flush is needed), x on
[-1, 1], y a random cubic plus N(0, 0.01^2) noise.  A step streams the points
once accumulating the degree-3 power sums (compensated FP32 accumulation,
FP64 cross-block combine) and solves the normal equations for m = 3, 2 and 1
from those sums (FP64 Gaussian elimination).  The metric is fitted points per
second; the roofline is that of the streaming kernel (8 algorithmic bytes per
point) against the measured HBM copy bandwidth.

Other workloads (--workload) are measured the same way and documented with
the library; the default line is the one the contract reports.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lsefit|reference]

Under torchrun each rank fits its own independent series (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fitted points/s (fwd)"
UNIT = "points/s"


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["lsefit", "reference"], default="lsefit")
    p.add_argument("--workload", default="single_large",
                   choices=["single_large", "ragged_batch", "diff_batch", "single_fp64", "general", "solve"])
    p.add_argument("--kind", default="weighted", choices=["weighted", "chebyshev", "weighted_chebyshev", "chebyshev16"],
                   help="objective of the general workload")
    p.add_argument("--n", type=int, default=1 << 28, help="points of the single_large series")
    p.add_argument("--series", type=int, default=65536, help="series of the ragged_batch workload")
    p.add_argument("--no-plain", action="store_true", help="skip the plain per-series comparison")
    p.add_argument("--coef-sample", type=int, default=2048,
                   help="series of a batch checked against the oracle after the timed region")
    p.add_argument("--no-coef", action="store_true",
                   help="general workload: skip the oracle check of the timed coefficients")
    p.add_argument("--no-sub", action="store_true",
                   help="default workload: skip the ragged and differentiable sub-records")
    p.add_argument("--tuning", default=None,
                   help="batched schedule as JSON (e.g. '{\"warp_max_len\": 1048576}'); default: autotune")
    p.add_argument("--accum", default="comp", choices=["comp", "naive", "f64"])
    p.add_argument("--basis", default="monomial", choices=["monomial", "chebyshev"],
                   help="basis of the ragged_batch fit (chebyshev: no plain per-series comparison)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=6.0,
                   help="target CPU time of the oracle baseline sample")
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; no collective on the data path)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, gpus: int):
        import torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if torch.cuda.is_available():
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist
        elif torch.cuda.is_available():
            torch.cuda.set_device(0)

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, v: float) -> float:
        return self.reduce(v, "max")

    def sum(self, v: float) -> float:
        return self.reduce(v, "sum")

    def reduce(self, v: float, op: str) -> float:
        if self.pg is None:
            return v
        import torch
        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else torch.device("cpu")
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Sources each recorded kernel is built from (traffic.json key prefix -> files
# of paper_1512_08017_gb300/csrc besides the shared ones); other keys hash
# every source file.
_SHARED_SOURCES = ("lsefit_device.cuh", "lsefit_host.h", "lsefit_api.cu")
_KERNEL_SOURCES = {
    "powersums": ("lsefit_powersums.cu",),
    "batched": ("lsefit_batched.cuh", "lsefit_batched.cu", "lsefit_batched_*.cu"),
    "residuals": ("lsefit_residuals.cu",),
    "general": ("lsefit_general.cuh", "lsefit_general.cu", "lsefit_general_*.cu"),
    "diff": ("lsefit_batched.cuh", "lsefit_batched.cu", "lsefit_batched_*.cu", "lsefit_backward.cu"),
}


def source_digest(kernel_key: str | None = None) -> str:
    """Hash of the CUDA sources a kernel is built from, plus the C header (ties a
    recorded ncu traffic figure to the code it was captured on).  Without a key,
    or for an unknown one, every source file."""
    import fnmatch
    csrc = os.path.join(ROOT, "paper_1512_08017_gb300", "csrc")
    names = sorted(os.listdir(csrc))
    prefix = (kernel_key or "").split("_")[0]
    if prefix in _KERNEL_SOURCES:
        pats = _SHARED_SOURCES + _KERNEL_SOURCES[prefix]
        names = [n for n in names if any(fnmatch.fnmatch(n, p) for p in pats)]
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    with open(os.path.join(ROOT, "include", "lsefit.h"), "rb") as f:
        h.update(b"lsefit.h")
        h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str):
    """DRAM bytes per launch from profiles/traffic.json if taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel_key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_digest") != source_digest(kernel_key):
        return None
    return rec.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, single thread, on a bounded sample
# ---------------------------------------------------------------------------
def host_info() -> dict:
    """Host cores and CPU model of the machine the oracle is timed on."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                fields.setdefault(key.strip(), val.strip())
    except OSError:
        pass
    # x86 names the model; Arm kernels give the implementer and part numbers
    model = fields.get("model name") or fields.get("Model")
    if not model and "CPU part" in fields:
        model = f"implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": model}


def cpu_baseline_single(x: np.ndarray, y: np.ndarray, m: int, target_s: float):
    """The oracle on the host cores, two ways: the sequential oracle itself (one
    thread, on the first 2^24 points) and its all-core variant (per-thread power
    sums over fixed equal point ranges, added in thread order, on every point);
    both then solve degrees m..1 by the oracle's elimination.  The all-core
    figure is the line's value."""
    import oracle
    n = x.size
    sample = min(n, 1 << 24)
    xs = x[:sample].astype(np.float64)
    ys = y[:sample].astype(np.float64)
    oracle.fit(xs[:1024], ys[:1024], m)  # build/load outside the timing
    reps, t_total = 0, 0.0
    while reps < 3 or t_total < target_s:
        t0 = time.perf_counter()
        out = oracle.fit(xs, ys, m)
        for k in range(m - 1, 0, -1):
            oracle.solve(out["S"][: 2 * k + 1], out["T"][: k + 1], k)
        t_total += time.perf_counter() - t0
        reps += 1
        if reps >= 1000:
            break
    assert out["status"] == "ok"
    single = {"value": sample * reps / t_total, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"first {sample} points of the series, degrees {m}..1 (FP64 sums + Gaussian elimination, "
                        f"sequential C), {reps} repetitions, {t_total:.1f} s"}
    del xs, ys
    threads = oracle.host_threads()
    x64 = x.astype(np.float64)
    y64 = y.astype(np.float64)
    reps, t_total = 0, 0.0
    while reps < 2 or t_total < max(1.0, target_s / 3):
        t0 = time.perf_counter()
        out = oracle.fit_threads(x64, y64, m, threads=threads)
        for k in range(m - 1, 0, -1):
            oracle.solve(out["S"][: 2 * k + 1], out["T"][: k + 1], k)
        t_total += time.perf_counter() - t0
        reps += 1
        if reps >= 200:
            break
    assert out["status"] == "ok"
    return {"value": n * reps / t_total, "unit": UNIT, "cores": threads, "kind": "oracle", "host": host_info(),
            "sample": f"all {n} points, degrees {m}..1: FP64 power sums on {threads} threads (fixed equal point "
                      f"ranges, the sequential oracle per range, added in thread order) + the oracle's Gaussian "
                      f"elimination; {reps} repetitions, {t_total:.1f} s",
            "single_thread": single}


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def coef_err_general(out, ref, m: int, accum: str, n: int, status: str) -> dict:
    """Error of the timed general fit of degree m (row m - 1 of the outputs, m_lo =
    1; status: its name) against the oracle's fit of the same stored points: relative errors of the
    basis and monomial coefficients, the normwise backward error of Xb in the
    oracle's G Xb = b, cond(G), and the gates the parity tests apply (forward:
    max(base, cond eps 4m) while at most 1e-3; backward: 1e-5 compensated, 1e-12 +
    2n 2^-53 FP64)."""
    rec = {"degree": m, "status": status, "oracle_status": ref["status"]}
    if rec["status"] != "ok" or ref["status"] != "ok":
        return rec
    Xb = np.asarray(out["Xb"][m - 1][: m + 1], dtype=np.float64)
    X = np.asarray(out["X"][m - 1][: m + 1], dtype=np.float64)
    G = np.asarray(ref["G"], dtype=np.float64)
    b = np.asarray(ref["b"], dtype=np.float64)
    cond = float(np.linalg.cond(G))
    eps, base = (2.0 ** -53, 1e-6) if accum == "f64" else (2.0 ** -24, 1e-5)
    fwd_gate = max(base, cond * eps * 4 * m)
    rec.update({
        "rel_Xb": rel_err(Xb, ref["Xb"]), "rel_X": rel_err(X, ref["X"]),
        "backward": float(np.linalg.norm(G @ Xb - b) / (np.linalg.norm(G, 2) * np.linalg.norm(Xb) + np.linalg.norm(b))),
        "cond_G": cond,
        "forward_gate": fwd_gate if fwd_gate <= 1e-3 else None,
        "backward_gate": 1e-12 + 2.0 * n * 2.0 ** -53 if accum == "f64" else (1e-3 if accum == "naive" else 1e-5),
    })
    return rec


def backward_err(S, T, m, Xt) -> float:
    """Normwise backward error of Xt in the oracle's normal equations A Xt = B
    (A[j][k] = S[j+k], B = T): the smallest relative change of A and B that makes
    Xt exact; it does not grow with cond(A)."""
    A = np.array([[S[j + k] for k in range(m + 1)] for j in range(m + 1)], dtype=np.float64)
    B = np.asarray(T[: m + 1], dtype=np.float64)
    Xt = np.asarray(Xt, dtype=np.float64)
    return float(np.linalg.norm(A @ Xt - B) / (np.linalg.norm(A, 2) * np.linalg.norm(Xt) + np.linalg.norm(B)))


def coef_err_single(x: np.ndarray, y: np.ndarray, out: dict, m: int, m_lo: int = 1, accum: str = "comp") -> dict:
    """Error of the timed single-series result (every degree m_lo..m, no interval)
    against the sequential FP64 oracle on all the stored points (singular
    threshold of the accumulation)."""
    import oracle
    eps = oracle.EPS64 if accum == "f64" else oracle.EPS32
    t0 = time.perf_counter()
    ref = oracle.fit(x.astype(np.float64), y.astype(np.float64), m, eps=eps)
    X = out["X"].cpu().numpy()
    Xt = out["Xt"].cpu().numpy()
    per = []
    for r, d in enumerate(range(m_lo, m + 1)):
        st, Xo = oracle.solve(ref["S"][: 2 * d + 1], ref["T"][: d + 1], d, eps=eps)
        per.append({"m": d, "status": st, "X": rel_err(X[r, : d + 1], Xo), "Xt": rel_err(Xt[r, : d + 1], Xo),
                    "backward": backward_err(ref["S"], ref["T"], d, Xt[r, : d + 1])})
    return {"max_rel_X": max(p["X"] for p in per), "max_rel_Xt": max(p["Xt"] for p in per),
            "max_backward": max(p["backward"] for p in per), "per_degree": per,
            "tolerance": 1e-6 if accum == "f64" else 1e-5,
            "oracle": f"sequential FP64 oracle on all {x.size} stored points",
            "oracle_s": time.perf_counter() - t0}


# ---------------------------------------------------------------------------
# host link: rate of one large pinned copy and where the buffers sit
# ---------------------------------------------------------------------------
_SYS_MOVE_PAGES = {"x86_64": 279, "aarch64": 239}


def page_node(addr: int):
    """NUMA node of the page holding host address addr (move_pages(2) query,
    no move), or None where the kernel does not say."""
    import ctypes
    import platform
    nr = _SYS_MOVE_PAGES.get(platform.machine())
    if nr is None:
        return None
    try:
        libc = ctypes.CDLL(None, use_errno=True)
        pages = (ctypes.c_void_p * 1)(addr & ~4095)
        status = (ctypes.c_int * 1)(-1)
        rc = libc.syscall(ctypes.c_long(nr), ctypes.c_int(0), ctypes.c_ulong(1), pages, None, status,
                          ctypes.c_int(0))
    except (OSError, AttributeError):
        return None
    return int(status[0]) if rc == 0 and status[0] >= 0 else None


def gpu_numa_node(device_index: int):
    """NUMA node the GPU's PCI function reports (sysfs), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(device_index), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True, timeout=20).stdout.strip()
    except (OSError, subprocess.TimeoutExpired):
        return None
    if not out:
        return None
    dom, rest = out.split(":", 1)
    for name in (f"{int(dom, 16):04x}:{rest}".lower(), out.lower()):
        try:
            with open(f"/sys/bus/pci/devices/{name}/numa_node") as f:
                return int(f.read().strip())
        except (OSError, ValueError):
            continue
    return None


def numa_nodes_with_cpus():
    base = "/sys/devices/system/node"
    nodes = {}
    try:
        for name in sorted(os.listdir(base)):
            if name.startswith("node") and name[4:].isdigit():
                with open(os.path.join(base, name, "cpulist")) as f:
                    nodes[int(name[4:])] = f.read().strip()
    except OSError:
        pass
    return nodes


def link_probe(host: "torch.Tensor", dev: "torch.Tensor", stream, reps: int = 3) -> dict:
    """Best H2D and D2H GB/s of one copy of the whole pinned buffer, and where
    the buffer and the GPU sit."""
    import torch
    h2d = d2h = 0.0
    nbytes = host.numel() * host.element_size()
    for _ in range(reps):
        for direction in ("h2d", "d2h"):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if direction == "h2d":
                dev.copy_(host, non_blocking=True)
            else:
                host.copy_(dev, non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            gbs = nbytes / (a.elapsed_time(b) / 1e3) / 1e9
            if direction == "h2d":
                h2d = max(h2d, gbs)
            else:
                d2h = max(d2h, gbs)
    return {"h2d_gbs": h2d, "d2h_gbs": d2h, "bytes": nbytes, "pinned_node": page_node(host.data_ptr()),
            "gpu_node": gpu_numa_node(torch.cuda.current_device()), "nodes_with_cpus": numa_nodes_with_cpus()}


# ---------------------------------------------------------------------------
# single_large: one long FP32 series
# ---------------------------------------------------------------------------
def run_single_large(args, dist: Dist):
    import torch
    import synth
    import paper_1512_08017_gb300 as L

    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.n
    m = 3
    # each rank draws its own series (seed offset by rank)
    hx = torch.empty(n, dtype=torch.float32).pin_memory()
    hy = torch.empty(n, dtype=torch.float32).pin_memory()
    d = synth.single_large(n=n, m=m, seed=synth.SEED_SINGLE_LARGE + dist.rank,
                           out_x=hx.numpy(), out_y=hy.numpy())
    x = hx.to(dev)
    y = hy.to(dev)
    stream = torch.cuda.current_stream()
    out = L.fit_degrees(x, y, m, 1, args.accum)  # allocates the outputs once

    def step(ev_pair=None):
        if ev_pair is not None:
            ev_pair[0].record(stream)
        L.fit_degrees(x, y, m, 1, args.accum, out=out)
        if ev_pair is not None:
            ev_pair[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of what is being timed (against the oracle) is the tests' job;
    # here only the status is checked.
    assert out["status"].tolist() == [L.OK] * 3

    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        step(kev[i])
    t1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in kev)
    ms_max = dist.max(ms)
    kern_ms_max = dist.max(kern_ms)

    # end to end through the same C ABI with host buffers: H2D copy of the step's
    # points from pinned memory, the fit, and the D2H read of the coefficients.
    e2e = None
    if not args.no_e2e:
        hX = torch.empty(4, dtype=torch.float64).pin_memory()  # the degree-3 coefficients
        e_steps = max(3, min(args.steps, 10))

        def e2e_step():
            x.copy_(hx, non_blocking=True)
            y.copy_(hy, non_blocking=True)
            step()
            hX.copy_(out["X"][2], non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = dist.max(e0.elapsed_time(e1))
        copy_mode = {"value": dist.world * n * e_steps / (e_ms / 1e3), "ms_per_step": e_ms / e_steps,
                     "desc": "cudaMemcpyAsync of x, y from pinned host memory, then the fit"}

        # the same call on the pinned host buffers themselves: the kernel streams
        # them over the CPU-GPU link (no staging copy)
        def e2e_mapped():
            L.fit_degrees(hx, hy, m, 1, args.accum, out=out)
            hX.copy_(out["X"][2], non_blocking=True)

        for _ in range(2):
            e2e_mapped()
        torch.cuda.synchronize()
        dist.barrier()
        em_total = _event_steps(e2e_mapped, e_steps, stream)
        em_ms = dist.max(em_total)
        mapped_mode = {"value": dist.world * n * e_steps / (em_ms / 1e3), "ms_per_step": em_ms / e_steps,
                       "desc": "lsefit_fit on the pinned host buffers (the kernel reads host memory)"}
        best = mapped_mode if mapped_mode["value"] > copy_mode["value"] else copy_mode
        e2e = {"value": best["value"], "unit": UNIT,
               "h2d_bytes_per_step": 2 * n * 4, "d2h_bytes_per_step": 4 * 8,
               "steps": e_steps, "ms_per_step": best["ms_per_step"],
               "mode": "mapped" if best is mapped_mode else "copy", "copy": copy_mode, "mapped": mapped_mode,
               "link": link_probe(hx, x, stream)}

    peaks, peak_kind = measured_peaks()
    algo_bytes = 8 * n
    achieved = algo_bytes / (kern_ms_max / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": recorded_traffic("powersums_f32_comp_m3"),
                "kernel": "ps_kernel_f32<3,F32,comp> (fused solves of degrees 1-3)", "kernel_ms": kern_ms_max,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6800 GB/s"}
    # error of the timed result against the oracle on every stored point (after the timed region)
    coef = coef_err_single(d["x"], d["y"], out, m) if dist.rank == 0 else None
    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_single(d["x"], d["y"], m, args.cpu_seconds)
    value = dist.world * n * args.steps / (ms_max / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; x ~ U[-1,1], y = random cubic + N(0, 0.01^2))",
        "config": {"workload": "single series, n=2^28 FP32 points (2 GiB), degrees 3,2,1 from one pass",
                   "n": n, "m": [3, 2, 1], "accum": args.accum, "solve": "fp64 GE, partial pivoting",
                   "l2": "inputs (2 GiB) larger than L2; no flush", "parallelism": f"replicas x{dist.world}"},
        "hbm_gbs": algo_bytes / (ms_max / args.steps / 1e3) / 1e9,
        "roofline": roofline, "coef_err": coef, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "gpu_launches": args.steps,
    }
    return line


# ---------------------------------------------------------------------------
# shared timing helpers for the batched workloads
# ---------------------------------------------------------------------------
def _event_steps(step, steps, stream):
    """Device time (ms) of `steps` back-to-back calls of step(), between one pair of
    CUDA events on `stream`.  (An event pair around every call adds about 4 us per
    step: the records separate consecutive graph launches.)"""
    import torch
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1)


def _graph(fn, stream):
    """Capture fn() (after one warm call on a side stream) into a CUDA graph."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        fn()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def _roofline(algo_bytes, kern_ms, kernel, key):
    peaks, peak_kind = measured_peaks()
    achieved = algo_bytes / (kern_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": recorded_traffic(key), "kernel": kernel,
            "kernel_ms": kern_ms,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6800 GB/s"}


def _roofline_fp64(flops, kern_ms, kernel):
    """FP64-bound kernels: achieved GFLOP/s against the nominal FP64 rate (the
    measured peaks cover HBM and bf16 only).  flops counts each FMA as two."""
    achieved = flops / (kern_ms / 1e3) / 1e9
    return {"bound": "fp64", "achieved": achieved, "peak": 1250.0, "unit": "GFLOP/s", "frac": achieved / 1250.0,
            "traffic": None, "kernel": kernel, "kernel_ms": kern_ms,
            "peak_source": "nominal FP64 1.25 TFLOP/s (no measured FP64 figure)"}


def coef_err_batched(b: dict, res: dict, series, basis: str = "monomial", accum: str = "comp") -> dict:
    """Error of a batched result on the given series against the sequential
    oracle (same stored points, same map): statuses, the normwise error of the
    mapped-basis coefficients where the system determines them to 1e-3 or
    better (cond(A) 2^-24 4m <= 1e-3), and the backward error everywhere."""
    import oracle
    t0 = time.perf_counter()
    Xt = res["Xt"].cpu().numpy()
    st = res["status"].cpu().numpy()
    names = {0: "ok", 2: "n_too_small", 3: "singular", 4: "nonfinite", 5: "bad_interval"}
    x64 = b["x"]
    y64 = b["y"]
    fwd_max, bwd_max, mismatched, undetermined, checked = 0.0, 0.0, 0, 0, 0
    for s_ in series:
        lo, hi = int(b["offsets"][s_]), int(b["offsets"][s_ + 1])
        m = int(b["degree"][s_])
        xs = x64[lo:hi].astype(np.float64)
        ys = y64[lo:hi].astype(np.float64)
        if basis == "monomial":
            r = oracle.fit_interval(xs, ys, m, *b["interval"][s_], fp32=accum != "f64")
            ref, A, B = r["Xt"], (None if r["S"] is None else
                                  np.array([[r["S"][j + k] for k in range(m + 1)] for j in range(m + 1)])), r["T"]
        else:
            r = oracle.fit_general_interval(xs, ys, m, *b["interval"][s_], fp32=accum != "f64", basis="chebyshev")
            ref, A, B = r["Xb"], r["G"], r["b"]
        if names.get(int(st[s_]), "other") != r["status"]:
            mismatched += 1
            continue
        if r["status"] != "ok":
            continue
        checked += 1
        got = Xt[s_, : m + 1]
        eta = float(np.linalg.norm(A @ got - B) / (np.linalg.norm(A, 2) * np.linalg.norm(got) + np.linalg.norm(B)))
        bwd_max = max(bwd_max, eta)
        cond = float(np.linalg.cond(A))
        eps = 2.0 ** -53 if accum == "f64" else 2.0 ** -24
        if cond * eps * 4 * m <= 1e-3:
            fwd_max = max(fwd_max, rel_err(got, ref))
        else:
            undetermined += 1
    return {"series_checked": checked, "status_mismatches": mismatched, "max_rel_Xt": fwd_max,
            "max_backward": bwd_max, "undetermined_reported": undetermined,
            "oracle": f"sequential FP64 oracle per series ({basis} basis)", "oracle_s": time.perf_counter() - t0}


# ---------------------------------------------------------------------------
# ragged_batch: 65,536 independent series of uneven length and mixed degree
# ---------------------------------------------------------------------------
def run_ragged_batch(args, dist: Dist):
    import ctypes
    import torch
    import synth
    import paper_1512_08017_gb300 as L
    from paper_1512_08017_gb300 import autotune, lsefit as B

    dev = torch.device("cuda", torch.cuda.current_device())
    b = synth.ragged_batch(num_series=args.series, seed=synth.SEED_RAGGED + dist.rank)
    S = len(b["degree"])
    N = int(b["offsets"][-1])
    m_max = 5
    hx = torch.from_numpy(b["x"]).pin_memory()
    hy = torch.from_numpy(b["y"]).pin_memory()
    x, y = hx.to(dev), hy.to(dev)
    off = torch.from_numpy(b["offsets"]).to(dev)
    deg = torch.from_numpy(b["degree"]).to(dev)
    iv = torch.from_numpy(b["interval"]).to(dev)
    t_tune = time.perf_counter()
    if args.tuning:
        tuning, tried = json.loads(args.tuning), []
    else:
        tuning, tried = autotune.tune_batched(x, y, off, deg, iv, m_max=m_max, accum=args.accum, basis=args.basis)
    t_tune = time.perf_counter() - t_tune
    t_plan = time.perf_counter()
    plan = L.BatchPlan(b["offsets"], m_max, tuning=tuning, device=dev, degree=b["degree"])
    t_plan = time.perf_counter() - t_plan
    out = {"X": torch.empty(S, m_max + 1, dtype=torch.float64, device=dev),
           "status": torch.empty(S, dtype=torch.int32, device=dev)}
    stream = torch.cuda.current_stream()

    def fwd():
        L.fit_batched(x, y, off, deg, iv, m_max=m_max, accum=args.accum, plan=plan, out=out, basis=args.basis)

    g = _graph(fwd, stream)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    assert int((out["status"] != 0).sum().item()) == 0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    total = _event_steps(g.replay, args.steps, stream)
    dist.barrier()
    clk = clocks.stop()
    ms = dist.max(total)
    step_ms = dist.max(total / args.steps)
    per_series_bytes = 8 + 4 + 16 + 8 * (m_max + 1) + 4
    algo = 8 * N + per_series_bytes * S

    # plain per-series path: one single-series fit launch per series from a host loop
    plain = None
    if not args.no_plain and args.basis == "monomial":
        wsz = L.lib.lsefit_powersums_workspace_size(m_max)
        ws = torch.zeros(wsz, dtype=torch.uint8, device=dev)
        Xp = torch.empty(S, m_max + 1, dtype=torch.float64, device=dev)
        stp = torch.empty(S, dtype=torch.int32, device=dev)
        fn = B.lib.lsefit_fit
        xs, ys, ivp = x.data_ptr(), y.data_ptr(), iv.data_ptr()
        sh = ctypes.c_void_p(stream.cuda_stream)
        calls = []
        for s_ in range(S):
            lo, hi = int(b["offsets"][s_]), int(b["offsets"][s_ + 1])
            m = int(b["degree"][s_])
            calls.append((ctypes.c_void_p(xs + 4 * lo), ctypes.c_void_p(ys + 4 * lo), hi - lo, B.F32, m, m,
                          B.ACCUM[args.accum], ctypes.c_void_p(ivp + 16 * s_),
                          ctypes.c_void_p(Xp.data_ptr() + 8 * (m_max + 1) * s_), None, None, None,
                          ctypes.c_void_p(stp.data_ptr() + 4 * s_), ctypes.c_void_p(ws.data_ptr()), wsz, sh))

        def plain_step():
            for c_ in calls:
                fn(*c_)

        plain_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)
        plain_step()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        pms = e0.elapsed_time(e1)
        plain = {"value": N / (pms / 1e3), "unit": UNIT, "ms_per_step": pms, "host_wall_s": wall,
                 "launches_per_step": S, "desc": "one lsefit_fit launch per series from a host loop, no graph"}

    # the residual/SSE pass over the same batch (reads x, y once more: 8 B/point),
    # from a fit that also keeps the mapped-basis coefficients and the map
    residuals = None
    fwd_full = L.fit_batched(x, y, off, deg, iv, m_max=m_max, accum=args.accum, plan=plan, basis=args.basis)
    res_out = L.residuals_batched(x, y, off, deg, fwd_full)
    torch.cuda.synchronize()
    coef = None
    if dist.rank == 0:
        # the timed graph's coefficients are these, bit for bit; a sample of series
        # (and the longest and shortest) against the oracle
        same = bool(torch.equal(torch.nan_to_num(fwd_full["X"]), torch.nan_to_num(out["X"])))
        rng = np.random.default_rng(11)
        lens = np.diff(b["offsets"])
        pick = sorted(set(rng.choice(S, min(S, args.coef_sample), replace=False).tolist())
                      | {int(np.argmax(lens)), int(np.argmin(lens))})
        coef = coef_err_batched(b, fwd_full, pick, args.basis, args.accum)
        coef["timed_result_identical"] = same
    assert bool(torch.isfinite(res_out["sse"]).all())
    rtot = _event_steps(lambda: L.residuals_batched(x, y, off, deg, fwd_full), args.steps, stream)
    r_ms = dist.max(rtot / args.steps)
    cheb = args.basis != "monomial"
    residuals = {"ms_per_step": r_ms, "hbm_gbs": 8 * N / (r_ms / 1e3) / 1e9,
                 "roofline": _roofline(8 * N, r_ms,
                                       "residuals_kernel<F32{}> (+ prep launch)".format(",chebyshev" if cheb else ""),
                                       "residuals_f32_chebyshev" if cheb else "residuals_f32"),
                 "desc": "lsefit_residuals: SSE and V^T r per series from the fit's Xt and map"
                         + (" (Clenshaw evaluation, T_k(t) r diagnostics)" if cheb else "")}

    e2e = None
    if not args.no_e2e:
        hX = torch.empty(S, m_max + 1, dtype=torch.float64).pin_memory()

        def e2e_step():
            x.copy_(hx, non_blocking=True)
            y.copy_(hy, non_blocking=True)
            g.replay()
            hX.copy_(out["X"], non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e_total = _event_steps(e2e_step, 3, stream)
        e_ms = dist.max(e_total) / 3
        e2e = {"value": dist.world * N / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": 8 * N,
               "d2h_bytes_per_step": 8 * (m_max + 1) * S, "ms_per_step": e_ms}

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        import oracle
        rng = np.random.default_rng(7)
        pick = rng.choice(S, min(S, 3000), replace=False)
        pts = 0
        t0 = time.perf_counter()
        for s_ in pick:
            lo, hi = int(b["offsets"][s_]), int(b["offsets"][s_ + 1])
            r = oracle.fit_interval(b["x"][lo:hi], b["y"][lo:hi], int(b["degree"][s_]), *b["interval"][s_],
                                    fp32=True)
            pts += hi - lo
        dt = time.perf_counter() - t0
        cpu = {"value": pts / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
               "sample": f"{len(pick)} random series of the batch ({pts} points), oracle fit per series, "
                         f"{dt:.1f} s"}
    return {
        "metric": "fitted points/s (fwd, batched ragged)", "value": dist.world * N * args.steps / (ms / 1e3),
        "unit": UNIT, "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ragged batch)",
        "config": {"workload": f"batched ragged: {S} series, lengths log-uniform 16..65536, degrees 1..5, "
                               "per-series intervals; one persistent launch in a CUDA graph",
                   "series": S, "points": N, "accum": args.accum, "basis": args.basis, "tuning": tuning,
                   "autotune_s": t_tune, "plan_build_s": t_plan, "autotune_candidates": len(tried),
                   "l2": f"inputs ({8 * N / 1e9:.1f} GB) larger than L2; no flush"},
        "hbm_gbs": algo / (step_ms / 1e3) / 1e9,
        "roofline": _roofline(algo, step_ms,
                              "batched_kernel<5,F32,{}{}> (+ prep launch)".format(
                                  args.accum, ",chebyshev" if args.basis != "monomial" else ""),
                              "batched_f32_comp" if args.basis == "monomial" else "batched_f32_comp_chebyshev"),
        "plain_per_series": plain,
        "speedup_vs_plain": (plain["ms_per_step"] / (ms / args.steps)) if plain else None,
        "coef_err": coef, "residuals": residuals,
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": 2 * args.steps,
    }


# ---------------------------------------------------------------------------
# diff_batch: 4,096 series x 4,096 points, forward + hand-written backward
# ---------------------------------------------------------------------------
def run_diff_batch(args, dist: Dist):
    import ctypes
    import torch
    import synth
    import paper_1512_08017_gb300 as L
    from paper_1512_08017_gb300 import lsefit as B

    dev = torch.device("cuda", torch.cuda.current_device())
    d = synth.diff_batch(seed=synth.SEED_DIFF + dist.rank)
    S, n = d["x"].shape
    N = S * n
    m = 3
    x = torch.from_numpy(d["x"].reshape(-1)).to(dev)
    y = torch.from_numpy(d["y"].reshape(-1)).to(dev)
    offsets = np.arange(S + 1, dtype=np.int64) * n
    off = torch.from_numpy(offsets).to(dev)
    deg = torch.full((S,), m, dtype=torch.int32, device=dev)
    iv = torch.tensor([[-1.0, 1.0]] * S, dtype=torch.float64, device=dev)
    w = torch.from_numpy(d["w"]).to(dev)
    from paper_1512_08017_gb300 import autotune
    if args.tuning:
        tuning = json.loads(args.tuning)
    else:
        tuning, _ = autotune.tune_batched(x, y, off, deg, iv, m_max=m, accum=args.accum)
    plan = L.BatchPlan(offsets, m, tuning=tuning, device=dev, degree=deg)
    fwd_out = {"X": torch.empty(S, m + 1, dtype=torch.float64, device=dev),
               "Xt": torch.empty(S, m + 1, dtype=torch.float64, device=dev),
               "sums": torch.empty(S, 3 * m + 2, dtype=torch.float64, device=dev),
               "map": torch.empty(S, 2, dtype=torch.float64, device=dev),
               "status": torch.empty(S, dtype=torch.int32, device=dev)}
    dx = torch.empty_like(x)
    dy = torch.empty_like(y)
    bst = torch.empty(S, dtype=torch.int32, device=dev)
    gX = torch.empty(S, m + 1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def fwd():
        L.fit_batched(x, y, off, deg, iv, m_max=m, accum=args.accum, plan=plan, out=fwd_out)

    w2 = 2.0 * w  # dL/dX of the user's loss L = sum w X^2 is 2 w X: one multiply per step

    def fwd_bwd():
        fwd()
        torch.mul(fwd_out["X"], w2, out=gX)
        L.backward(x, y, off, deg, fwd_out, gX, dx=dx, dy=dy, status=bst, accum=args.accum)

    gf = _graph(fwd, stream)
    gb = _graph(fwd_bwd, stream)
    for _ in range(args.warmup):
        gf.replay()
        gb.replay()
    torch.cuda.synchronize()
    assert int((bst != 0).sum().item()) == 0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    totf = _event_steps(gf.replay, args.steps, stream)
    dist.barrier()
    clk_f = clocks.stop()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    totb = _event_steps(gb.replay, args.steps, stream)
    dist.barrier()
    clk = clocks.stop()
    msf = dist.max(totf) / args.steps
    msb = dist.max(totb) / args.steps
    # errors of the timed results against the oracle: forward coefficients of a
    # sample of series, gradients of a few (the oracle's adjoint of its own fit)
    coef = None
    if dist.rank == 0:
        import oracle
        t0 = time.perf_counter()
        X = fwd_out["X"].cpu().numpy()
        Xt_all = fwd_out["Xt"].cpu().numpy()
        dxh = dx.cpu().numpy()
        dyh = dy.cpu().numpy()
        rng = np.random.default_rng(12)
        pick = sorted(rng.choice(S, min(S, 64), replace=False).tolist())
        fmax = bmax = gmax = 0.0
        for i, s_ in enumerate(pick):
            xs = d["x"][s_].astype(np.float64)
            ys = d["y"][s_].astype(np.float64)
            r = oracle.fit_interval(xs, ys, m, -1.0, 1.0, fp32=True)
            assert r["status"] == "ok"
            fmax = max(fmax, rel_err(Xt_all[s_], r["Xt"]), rel_err(X[s_], r["X"]))
            bmax = max(bmax, backward_err(r["S"], r["T"], m, Xt_all[s_]))
            if i < 8:
                st, odx, ody = oracle.backward(xs, ys, m, (r["c"], r["s"]), r["S"], r["Xt"], 2.0 * d["w"][s_] * r["X"])
                gmax = max(gmax, rel_err(dxh[s_ * n:(s_ + 1) * n], odx), rel_err(dyh[s_ * n:(s_ + 1) * n], ody))
        coef = {"series_checked": len(pick), "max_rel_Xt_X": fmax, "max_backward": bmax,
                "gradients_checked": min(8, len(pick)), "max_rel_dx_dy": gmax, "tolerance": {"X": 1e-5, "dx_dy": 1e-4},
                "oracle": "sequential FP64 oracle: fit and adjoint per series", "oracle_s": time.perf_counter() - t0}
    plain = None
    if not args.no_plain:
        # one single-series forward and one single-series backward launch pair per series
        plan1 = L.BatchPlan(np.array([0, n], dtype=np.int64), m, device=dev)
        wsz = L.lib.lsefit_powersums_workspace_size(m)
        ws = torch.zeros(wsz, dtype=torch.uint8, device=dev)
        bws = torch.zeros(L.lib.lsefit_backward_workspace_size(ctypes.byref(plan1.plan)), dtype=torch.uint8,
                          device=dev)
        off1 = torch.tensor([0, n], dtype=torch.int64, device=dev)
        deg1 = torch.tensor([m], dtype=torch.int32, device=dev)
        Xs = torch.empty(S, m + 1, dtype=torch.float64, device=dev)
        Xts = torch.empty(S, m + 1, dtype=torch.float64, device=dev)
        sums = torch.empty(S, 3 * m + 2, dtype=torch.float64, device=dev)
        mp = torch.empty(S, 2, dtype=torch.float64, device=dev)
        st = torch.empty(S, dtype=torch.int32, device=dev)
        sh = ctypes.c_void_p(stream.cuda_stream)
        batches = []
        for s_ in range(S):
            bb = B.Batch(x.data_ptr() + 4 * n * s_, y.data_ptr() + 4 * n * s_, off1.data_ptr(), deg1.data_ptr(),
                         None, 1, m, B.F32, B.ACCUM[args.accum], 0)
            batches.append(bb)

        def plain_step():
            for s_ in range(S):
                B.lib.lsefit_fit(ctypes.c_void_p(x.data_ptr() + 4 * n * s_), ctypes.c_void_p(y.data_ptr() + 4 * n * s_),
                                 n, B.F32, m, m, B.ACCUM[args.accum], ctypes.c_void_p(iv.data_ptr() + 16 * s_),
                                 ctypes.c_void_p(Xs.data_ptr() + 8 * (m + 1) * s_),
                                 ctypes.c_void_p(Xts.data_ptr() + 8 * (m + 1) * s_),
                                 ctypes.c_void_p(sums.data_ptr() + 8 * (3 * m + 2) * s_),
                                 ctypes.c_void_p(mp.data_ptr() + 16 * s_), ctypes.c_void_p(st.data_ptr() + 4 * s_),
                                 ctypes.c_void_p(ws.data_ptr()), wsz, sh)
            torch.mul(Xs, w2, out=gX)
            for s_ in range(S):
                B.lib.lsefit_backward(ctypes.byref(batches[s_]), ctypes.byref(plan1.plan),
                                      ctypes.c_void_p(sums.data_ptr() + 8 * (3 * m + 2) * s_),
                                      ctypes.c_void_p(Xts.data_ptr() + 8 * (m + 1) * s_),
                                      ctypes.c_void_p(mp.data_ptr() + 16 * s_),
                                      ctypes.c_void_p(gX.data_ptr() + 8 * (m + 1) * s_),
                                      ctypes.c_void_p(dx.data_ptr() + 4 * n * s_),
                                      ctypes.c_void_p(dy.data_ptr() + 4 * n * s_),
                                      ctypes.c_void_p(bst.data_ptr() + 4 * s_), ctypes.c_void_p(bws.data_ptr()),
                                      bws.numel(), sh)

        plain_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plain_step()
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": N / (pms / 1e3), "unit": UNIT, "ms_per_step": pms, "launches_per_step": 4 * S,
                 "desc": "per series: one lsefit_fit and one lsefit_backward call from a host loop, no graph"}
    e2e = None
    if not args.no_e2e:
        hx = torch.from_numpy(d["x"].reshape(-1)).pin_memory()
        hy = torch.from_numpy(d["y"].reshape(-1)).pin_memory()
        hdx = torch.empty(N, dtype=torch.float32).pin_memory()
        hdy = torch.empty(N, dtype=torch.float32).pin_memory()

        def e2e_step():
            x.copy_(hx, non_blocking=True)
            y.copy_(hy, non_blocking=True)
            gb.replay()
            hdx.copy_(dx, non_blocking=True)
            hdy.copy_(dy, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e_total = _event_steps(e2e_step, 3, stream)
        e_ms = dist.max(e_total) / 3
        e2e = {"value": dist.world * N / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": 8 * N,
               "d2h_bytes_per_step": 8 * N, "ms_per_step": e_ms}
    return {
        "metric": "fitted points/s (fwd+bwd)", "value": dist.world * N / (msb / 1e3), "unit": UNIT,
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": msb,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded)",
        "config": {"workload": "differentiable fit: 4096 series x 4096 FP32 points, degree 3, "
                               "L = sum w X^2; forward + backward in one CUDA graph",
                   "series": S, "points": N, "accum": args.accum, "tuning": plan.tuning},
        "fwd": {"value": dist.world * N / (msf / 1e3), "unit": UNIT, "ms_per_step": msf,
                "hbm_gbs": 8 * N / (msf / 1e3) / 1e9,
                "roofline": _roofline(8 * N, msf, "batched forward (8 B/point)", "diff_fwd"), "clocks": clk_f},
        "fwd_bwd_hbm_gbs": 24 * N / (msb / 1e3) / 1e9,
        "roofline": _roofline(24 * N, msb, "batched forward + lambda + grad kernels", "diff_fwd_bwd"),
        "plain_per_series": plain,
        "speedup_vs_plain": (plain["ms_per_step"] / msb) if plain else None,
        "coef_err": coef,
        "cpu_baseline": None, "e2e": e2e, "clocks": clk, "gpu_launches": 4 * args.steps,
    }


# ---------------------------------------------------------------------------
# solve: the normal equations of 65,536 degree-5 fits, by Gaussian elimination
# and by Cholesky factorisation (one system per thread, FP64)
# ---------------------------------------------------------------------------
def run_solve(args, dist: Dist):
    import torch
    import synth
    import paper_1512_08017_gb300 as L

    dev = torch.device("cuda", torch.cuda.current_device())
    m = 5
    b = synth.ragged_batch(num_series=args.series, seed=synth.SEED_RAGGED + dist.rank)
    S = len(b["degree"])
    deg = np.full(S, m, dtype=np.int32)
    x = torch.from_numpy(b["x"]).to(dev)
    y = torch.from_numpy(b["y"]).to(dev)
    fwd = L.fit_batched(x, y, b["offsets"], deg, b["interval"], m_max=m, accum="comp")
    torch.cuda.synchronize()
    sums, mp = fwd["sums"], fwd["map"]
    ok = fwd["status"] == 0
    stream = torch.cuda.current_stream()
    res = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for method in ("gauss", "cholesky"):
        X = torch.empty(S, m + 1, dtype=torch.float64, device=dev)
        Xt = torch.empty_like(X)
        st = torch.empty(S, dtype=torch.int32, device=dev)

        def step():
            L.solve(sums, m, map=mp, accum="comp", X=X, Xt=Xt, status=st, method=method)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        total = _event_steps(step, args.steps, stream)
        res[method] = {"ms": dist.max(total / args.steps), "Xt": Xt.clone(), "status": st.clone()}
    clk = clocks.stop()
    both = ok & (res["gauss"]["status"] == 0) & (res["cholesky"]["status"] == 0)
    a, c = res["gauss"]["Xt"][both], res["cholesky"]["Xt"][both]
    agree = float(((a - c).norm(dim=1) / a.norm(dim=1)).max().item())
    # the GPU elimination against the oracle's on the same FP64 sums, every system
    import oracle
    t0 = time.perf_counter()
    sh = sums.cpu().numpy()
    Xg = res["gauss"]["Xt"].cpu().numpy()
    stg = res["gauss"]["status"].cpu().numpy()
    okh = ok.cpu().numpy()
    worst = bmax = 0.0
    mism = 0
    for i in np.nonzero(okh)[0]:
        st_o, Xo = oracle.solve(sh[i, : 2 * m + 1], sh[i, 2 * m + 1: 3 * m + 2], m, eps=oracle.EPS32)
        if (st_o == "ok") != (stg[i] == 0):
            mism += 1
            continue
        if st_o == "ok":
            worst = max(worst, rel_err(Xg[i], Xo))
            bmax = max(bmax, backward_err(sh[i, : 2 * m + 1], sh[i, 2 * m + 1:], m, Xg[i]))
    coef = {"systems_checked": int(okh.sum()), "status_mismatches": mism, "max_rel_Xt": worst,
            "max_backward": bmax, "oracle": "the oracle's Gaussian elimination on the same FP64 sums",
            "oracle_s": time.perf_counter() - t0}
    n1 = m + 1
    flops = {"gauss": 2 * n1 ** 3 / 3 + 2 * n1 ** 2, "cholesky": n1 ** 3 / 3 + 2 * n1 ** 2}
    out = {}
    for k in res:
        ms = res[k]["ms"]
        out[k] = {"ms_per_launch": ms, "systems_per_s": S / (ms / 1e3),
                  "gflops": S * flops[k] / (ms / 1e3) / 1e9,
                  "singular": int((res[k]["status"] == 3).sum().item())}
    ms_g = out["gauss"]["ms_per_launch"]
    return {"metric": "normal-equation systems solved/s (degree 5, FP64 GE)", "value": out["gauss"]["systems_per_s"],
            "unit": "systems/s", "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_g, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (power sums of the seeded ragged batch fitted at degree 5)",
            "config": {"workload": f"{S} degree-5 normal-equation systems from one batched pass, "
                                   "one system per thread", "series": S, "m": m},
            "gauss": out["gauss"], "cholesky": out["cholesky"], "max_rel_diff_gauss_cholesky": agree,
            "coef_err": coef, "clocks": clk,
            "roofline": {"bound": "fp64 latency", "achieved": out["gauss"]["gflops"], "peak": 1250.0,
                         "unit": "GFLOP/s", "frac": out["gauss"]["gflops"] / 1250.0, "traffic": None,
                         "peak_source": "nominal FP64 (no measured FP64 figure)"},
            "gpu_launches": 2 * args.steps}


# ---------------------------------------------------------------------------
# single_fp64: the plain method on 100,000 FP64 points, degrees 1-3 in one launch
# ---------------------------------------------------------------------------
def run_single_fp64(args, dist: Dist):
    import torch
    import synth
    import paper_1512_08017_gb300 as L

    dev = torch.device("cuda", torch.cuda.current_device())
    d = synth.single_fp64(seed=synth.SEED_SINGLE_FP64 + dist.rank)
    n = d["x"].size
    x = torch.from_numpy(d["x"]).to(dev)
    y = torch.from_numpy(d["y"]).to(dev)
    out = L.fit_degrees(x, y, 3, 1, "f64")
    stream = torch.cuda.current_stream()
    g = _graph(lambda: L.fit_degrees(x, y, 3, 1, "f64", out=out), stream)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    total = _event_steps(g.replay, args.steps, stream)
    dist.barrier()
    clk = clocks.stop()
    ms = dist.max(total) / args.steps
    coef = coef_err_single(d["x"], d["y"], out, 3, 1, accum="f64") if dist.rank == 0 else None
    return {"metric": "fit latency (FP64, degrees 1-3 in one launch)", "clocks": clk, "value": ms * 1e3, "unit": "us",
            "coef_err": coef,
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "points_per_s": n / (ms / 1e3),
            "config": {"workload": "single series, n=100,000 FP64, x ~ U[0,10], degrees 1,2,3", "n": n},
            "gpu_launches": args.steps}


# ---------------------------------------------------------------------------
# general: the weighted and Chebyshev-basis fits of one long series
# ---------------------------------------------------------------------------
GENERAL_KINDS = {
    # kind: (weights, basis, degree, interval, description)
    "weighted": (True, "monomial", 3, (-1.0, 1.0),
                 "single series, n=2^28 FP32 points + FP32 weights (3 GiB), x ~ U[-1,1], w ~ U[0.1,3], "
                 "weighted degrees 3,2,1 from one pass"),
    "chebyshev": (False, "chebyshev", 8, (0.0, 1000.0),
                  "single series, n=2^28 FP32 points (2 GiB), x ~ U[0,1000] mapped to [-1,1], "
                  "Chebyshev basis, degrees 8..1 from one pass"),
    "weighted_chebyshev": (True, "chebyshev", 8, (0.0, 1000.0),
                           "single series, n=2^28 FP32 points + FP32 weights (3 GiB), x ~ U[0,1000] mapped, "
                           "weighted Chebyshev basis, degrees 8..1 from one pass"),
    "chebyshev16": (False, "chebyshev", 16, (0.0, 1000.0),
                    "single series, n=2^28 FP32 points (2 GiB), x ~ U[0,1000] mapped to [-1,1], "
                    "Chebyshev basis, degrees 16..1 from one pass (FP64 accumulation)"),
}


def cpu_baseline_general(x, y, w, m, basis, interval, target_s, fp32=True):
    import oracle
    n = x.size
    sample = min(n, 1 << 22)
    xs = x[:sample].astype(np.float64)
    ys = y[:sample].astype(np.float64)
    ws = w[:sample].astype(np.float64) if w is not None else None
    reps, t_total = 0, 0.0
    while reps < 3 or t_total < target_s:
        t0 = time.perf_counter()
        out = oracle.fit_general_interval(xs, ys, m, *interval, fp32=fp32, w=ws, basis=basis)
        t_total += time.perf_counter() - t0
        reps += 1
        if reps >= 1000:
            break
    assert out["status"] == "ok"
    return {"value": sample * reps / t_total, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
            "sample": f"first {sample} points of the series, degree {m} {basis} fit"
                      f"{' with weights' if w is not None else ''} (FP64 normal equations from their "
                      f"definition, sequential C), {reps} repetitions, {t_total:.1f} s"}


def run_general(args, dist: Dist):
    import torch
    import synth
    import paper_1512_08017_gb300 as L

    weighted, basis, m, interval, desc = GENERAL_KINDS[args.kind]
    accum = "f64" if m > 8 else args.accum  # degrees above 8: Chebyshev with FP64 accumulation
    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.n
    hx = torch.empty(n, dtype=torch.float32).pin_memory()
    hy = torch.empty(n, dtype=torch.float32).pin_memory()
    hw = torch.empty(n, dtype=torch.float32).pin_memory() if weighted else None
    d = synth.single_large(n=n, m=m, seed=synth.SEED_SINGLE_LARGE + dist.rank, out_x=hx.numpy(),
                           out_y=hy.numpy())
    lo, hi = interval
    if (lo, hi) != (-1.0, 1.0):  # the same polynomial of t, on x = lo + (t + 1) (hi - lo) / 2
        xn = hx.numpy()
        np.multiply(xn + np.float32(1.0), np.float32((hi - lo) / 2), out=xn)
        xn += np.float32(lo)
    if weighted:
        synth.weights(n, seed=synth.SEED_WEIGHTS + dist.rank, out=hw.numpy())
    x, y = hx.to(dev), hy.to(dev)
    w = hw.to(dev) if weighted else None
    stream = torch.cuda.current_stream()
    out = L.fit_general(x, y, m, w=w, basis=basis, m_lo=1, accum=accum, interval=interval)

    def step():
        L.fit_general(x, y, m, w=w, basis=basis, m_lo=1, accum=accum, interval=interval, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert out["status"].tolist() == [L.OK] * m
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    total = _event_steps(step, args.steps, stream)
    dist.barrier()
    clk = clocks.stop()
    timed = {k: out[k].cpu().numpy() for k in ("X", "Xb")}
    timed_status = L.status_names(out["status"])[m - 1]
    ms_max = dist.max(total)
    kern_ms = dist.max(total / args.steps)
    streams = 3 if weighted else 2
    algo_bytes = 4 * streams * n

    e2e = None
    if not args.no_e2e:
        hX = torch.empty(m + 1, dtype=torch.float64).pin_memory()
        e_steps = max(3, min(args.steps, 10))

        def e2e_step():
            x.copy_(hx, non_blocking=True)
            y.copy_(hy, non_blocking=True)
            if weighted:
                w.copy_(hw, non_blocking=True)
            step()
            hX.copy_(out["X"][m - 1], non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        dist.barrier()
        e_total = _event_steps(e2e_step, e_steps, stream)
        e_ms = dist.max(e_total)
        copy_mode = {"value": dist.world * n * e_steps / (e_ms / 1e3), "ms_per_step": e_ms / e_steps}

        def e2e_mapped():
            L.fit_general(hx, hy, m, w=hw, basis=basis, m_lo=1, accum=accum, interval=interval, out=out)
            hX.copy_(out["X"][m - 1], non_blocking=True)

        for _ in range(2):
            e2e_mapped()
        torch.cuda.synchronize()
        dist.barrier()
        em_total = _event_steps(e2e_mapped, e_steps, stream)
        em_ms = dist.max(em_total)
        mapped_mode = {"value": dist.world * n * e_steps / (em_ms / 1e3), "ms_per_step": em_ms / e_steps}
        best = mapped_mode if mapped_mode["value"] > copy_mode["value"] else copy_mode
        e2e = {"value": best["value"], "unit": UNIT,
               "h2d_bytes_per_step": streams * n * 4, "d2h_bytes_per_step": (m + 1) * 8,
               "steps": e_steps, "ms_per_step": best["ms_per_step"],
               "mode": "mapped" if best is mapped_mode else "copy", "copy": copy_mode, "mapped": mapped_mode}
    kname = "gen_kernel_{}<{},F32,{},W={},CHEB={}>".format("f64" if accum == "f64" else "f32", m, accum,
                                                          int(weighted), int(basis == "chebyshev"))
    coef = None
    if dist.rank == 0 and not args.no_coef:
        # the timed coefficients of degree m against the oracle on all n stored points
        import oracle
        t0 = time.perf_counter()
        ref = oracle.fit_general_interval(hx.numpy(), hy.numpy(), m, lo, hi, fp32=accum != "f64",
                                          w=hw.numpy() if weighted else None, basis=basis)
        coef = coef_err_general(timed, ref, m, accum, n, timed_status)
        coef.update({"oracle": f"sequential FP64 oracle (fit_general) on all {n} stored points; degrees "
                               f"{m - 1}..1 come from the same pass", "oracle_s": time.perf_counter() - t0})
    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_general(d["x"] if (lo, hi) == (-1.0, 1.0) else hx.numpy(), d["y"],
                                   hw.numpy() if weighted else None, m, basis, interval, args.cpu_seconds,
                                   fp32=accum != "f64")
    return {
        "metric": METRIC, "value": dist.world * n * args.steps / (ms_max / 1e3), "unit": UNIT,
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded)",
        "config": {"workload": desc, "n": n, "m": list(range(m, 0, -1)), "basis": basis, "weighted": weighted,
                   "accum": accum, "l2": "inputs larger than L2; no flush",
                   "parallelism": f"replicas x{dist.world}"},
        "roofline": _roofline(algo_bytes, kern_ms, kname, f"general_{args.kind}") if accum != "f64" else
        _roofline_fp64(n * (8 * m + 2 + (3 if weighted else 0)), kern_ms, kname),
        "coef_err": coef, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": args.steps,
    }


def run_reference(args, dist: Dist):
    """The oracle timed on the host cores on the same workload and metric: each
    step fits degrees 3, 2, 1 of the whole 2^28-point series, the power sums on
    all host cores (the sequential oracle per fixed point range, added in thread
    order), then the oracle's Gaussian elimination.  The sequential oracle alone
    is timed beside it on the first 2^24 points."""
    if dist.rank != 0:
        return None
    import synth
    import oracle
    m = 3
    n = args.n
    d = synth.single_large(n=n, m=m, seed=synth.SEED_SINGLE_LARGE)
    x64 = d["x"].astype(np.float64)
    y64 = d["y"].astype(np.float64)
    threads = oracle.host_threads()

    def step():
        out = oracle.fit_threads(x64, y64, m, threads=threads)
        for k in (2, 1):
            oracle.solve(out["S"][: 2 * k + 1], out["T"][: k + 1], k)
        return out

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = step()
    dt = time.perf_counter() - t0
    assert out["status"] == "ok"
    value = n * args.steps / dt
    sample = min(n, 1 << 24)
    t1 = time.perf_counter()
    reps = 0
    while reps < 2 or time.perf_counter() - t1 < 3.0:
        oracle.fit(x64[:sample], y64[:sample], m)
        reps += 1
    single = sample * reps / (time.perf_counter() - t1)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "single series, n=2^28 FP32 points (2 GiB), degrees 3,2,1 from one pass",
                       "n": n, "oracle_threads": threads},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "host": host_info(),
                             "sample": f"all {n} points per step: FP64 power sums on {threads} threads (the "
                                       f"sequential oracle per fixed point range), the oracle's elimination",
                             "single_thread": {"value": single, "unit": UNIT, "cores": 1,
                                               "sample": f"first {sample} points, sequential oracle, {reps} fits"}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


_SUB_KEYS = ("metric", "value", "unit", "ms_per_step", "config", "hbm_gbs", "roofline", "clocks", "fwd",
             "fwd_bwd_hbm_gbs", "plain_per_series", "speedup_vs_plain", "coef_err", "residuals", "e2e",
             "gpu_launches")


def run_default(args, dist: Dist):
    """The contract's line (the 2^28-point single series) with the rest of the
    metric as sub-records: the 65,536-series ragged batch (forward, CUDA graph,
    against the plain per-series path) and the differentiable 4,096 x 4,096
    batch (forward and forward + backward), each with its own roofline, clocks
    and coefficient error."""
    import torch
    line = run_single_large(args, dist)
    if args.no_sub:
        return line
    sub = argparse.Namespace(**vars(args))
    sub.no_cpu_baseline = True
    for key, runner in (("ragged", run_ragged_batch), ("diff", run_diff_batch)):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        rec = runner(sub, dist)
        line[key] = {k: rec[k] for k in _SUB_KEYS if k in rec}
    return line


def launch_local_ranks(n: int, argv) -> int:
    """`--gpus N` without a launcher: start N ranks of this script on this node
    (RANK, LOCAL_RANK, WORLD_SIZE and a free 127.0.0.1 port in each one's
    environment), wait for all, and return the first non-zero exit code."""
    import socket
    with socket.socket() as sock:
        sock.bind(("127.0.0.1", 0))
        port = sock.getsockname()[1]
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n), LOCAL_WORLD_SIZE=str(n),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), *argv], env=env))
    codes = [p.wait() for p in procs]
    bad = [c for c in codes if c != 0]
    return bad[0] if bad else 0


def main(argv=None):
    argv = list(sys.argv[1:] if argv is None else argv)
    args = parse_args(argv)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        if args.impl != "reference":
            import torch
            have = torch.cuda.device_count() if torch.cuda.is_available() else 0
            if have < args.gpus:
                print(f"bench.py: --gpus {args.gpus} asks for {args.gpus} ranks but this node has {have} GPU(s)",
                      file=sys.stderr)
                return 2
        return launch_local_ranks(args.gpus, argv)
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        line = run_reference(args, type("D", (), {"rank": 0, "world": world})())
        print(json.dumps(line))
        return 0
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    dist = Dist(args.gpus)
    try:
        runners = {"single_large": run_default, "ragged_batch": run_ragged_batch,
                   "diff_batch": run_diff_batch, "single_fp64": run_single_fp64, "general": run_general,
                   "solve": run_solve}
        line = runners[args.workload](args, dist)
        if dist.rank == 0 and line is not None:
            print(json.dumps(line))
    finally:
        dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
