"""Autotuner of the batched schedule.

The batched fit splits a batch into block tasks (long series, cut into
chunks) and warp tasks (short series).  The best split threshold, chunk
length and number of resident blocks depend on the length distribution and
on the device, so they are measured: each candidate plan is built, run a few
times with CUDA events around it, and the fastest is kept.  Results are
cached in a JSON file keyed by device name, SM count, storage type,
accumulation, maximum degree and a coarse signature of the layout (series
count, total points and the per-octave histogram of series lengths).
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np
import torch

from . import lsefit as L

DEFAULT_CANDIDATES = [
    {"warp_max_len": 1 << 20, "schedule": sched} for sched in (1, 2, 3)
] + [{"warp_max_len": wm, "chunk_len": ch, "schedule": 3}
     for wm in (4096, 65536) for ch in (65536, 262144)]

_lock = threading.Lock()


def cache_path() -> str:
    base = os.environ.get("LSEFIT_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "lsefit")
    return os.path.join(base, "autotune.json")


def layout_signature(offsets) -> str:
    off = L._as_host_int64(offsets)
    lens = np.diff(off)
    S = lens.size
    hist = np.bincount(np.floor(np.log2(np.maximum(lens, 1))).astype(np.int64), minlength=24)[:24]
    # coarse: counts rounded to 2 significant digits keep similar batches together
    coarse = [int(float(f"{h:.2g}")) if h else 0 for h in hist]
    total = int(off[-1]) if S else 0
    return f"S{S}:N{float(f'{total:.3g}'):g}:H{','.join(map(str, coarse))}"


def _key(device, dtype, accum, m_max, sig) -> str:
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|{p.multi_processor_count}|{dtype}|{accum}|m{m_max}|{sig}"


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def time_plan(x, y, offsets_d, degree_d, interval_d, m_max, accum, plan, reps=3, warmup=1) -> float:
    """Mean milliseconds of one fit_batched launch with `plan`."""
    out = None
    for _ in range(warmup):
        out = L.fit_batched(x, y, offsets_d, degree_d, interval_d, m_max=m_max, accum=accum, plan=plan, out=out)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        out = L.fit_batched(x, y, offsets_d, degree_d, interval_d, m_max=m_max, accum=accum, plan=plan, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batched(x, y, offsets, degree, interval=None, m_max=None, accum="comp", candidates=None, reps=3,
                 use_cache=True, verbose=False):
    """Best tuning dict for this batch layout (measured, or from the cache).

    Returns (tuning, results) where results lists (tuning, ms) per candidate
    measured now (empty when the cache answered)."""
    dev = x.device
    offsets_d = L._to_device(offsets, torch.int64, dev)
    degree_d = L._to_device(degree, torch.int32, dev)
    interval_d = L._to_device(interval, torch.float64, dev) if interval is not None else None
    if m_max is None:
        m_max = int(degree_d.max().item())
    off_host = L._as_host_int64(offsets)
    key = _key(dev, str(x.dtype), str(accum), m_max, layout_signature(off_host))
    with _lock:
        cache = _load_cache() if use_cache else {}
        if key in cache:
            return dict(cache[key]["tuning"]), []
    results = []
    for cand in candidates or DEFAULT_CANDIDATES:
        plan = L.BatchPlan(off_host, m_max, tuning=cand, device=dev, degree=degree)
        ms = time_plan(x, y, offsets_d, degree_d, interval_d, m_max, accum, plan, reps=reps)
        results.append((dict(cand), ms))
        if verbose:
            print(f"  tune {cand} -> {ms:.3f} ms")
    best, best_ms = min(results, key=lambda r: r[1])
    with _lock:
        cache = _load_cache() if use_cache else {}
        cache[key] = {"tuning": best, "ms": best_ms, "candidates": [[c, m] for c, m in results]}
        if use_cache:
            _store_cache(cache)
    return best, results
