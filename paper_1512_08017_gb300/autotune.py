"""Autotuner of the batched schedule (Python face of lsefit_plan_autotune).

The batched fit splits a batch into block tasks (long series, cut into
chunks) and warp tasks (short series), and warps draw their tasks in one of
three ways.  The best choice depends on the length and degree distribution
and on the device, so the library measures it: ``lsefit_plan_autotune``
builds each candidate plan, times it on the batch with CUDA events and
returns the fastest.  This module marshals that call and caches the answer in
a JSON file keyed by device name, SM count, CUDA driver version, storage
type, accumulation, basis, maximum degree and a coarse signature of the
layout (series count, total points and the per-octave histogram of series
lengths), so a tuning measured under another driver is measured again.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

import numpy as np
import torch

from . import lsefit as L

_lock = threading.Lock()


def builtin_candidates() -> list[dict]:
    """The library's built-in candidate tunings (lsefit_autotune_candidates)."""
    n = L.lib.lsefit_autotune_candidates(None, 0)
    arr = (L.Tuning * n)()
    L.lib.lsefit_autotune_candidates(arr, n)
    return [_tuning_dict(t) for t in arr]


def _tuning_dict(t) -> dict:
    return {"warp_max_len": t.warp_max_len, "chunk_len": t.chunk_len, "block_threads": t.block_threads,
            "blocks_per_sm": t.blocks_per_sm, "task_order": t.task_order, "schedule": t.schedule}


def _tuning_struct(d: dict):
    t = L.Tuning()
    for k, v in d.items():
        setattr(t, k, int(v))
    return t


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


def cache_key(device_name: str, num_sms: int, driver: int, dtype, accum, m_max: int, sig: str,
              basis: str = "monomial") -> str:
    return f"{device_name}|{num_sms}|drv{driver}|{dtype}|{accum}|{basis}|m{m_max}|{sig}"


def _device_key(device, dtype, accum, m_max, sig, basis) -> str:
    p = torch.cuda.get_device_properties(device)
    return cache_key(p.name, p.multi_processor_count, int(L.lib.lsefit_driver_version()), dtype, accum, m_max,
                     sig, basis)


def load_cache() -> dict:
    """The cache file's entries; an unreadable or malformed file counts as empty."""
    try:
        with open(cache_path()) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    if not isinstance(data, dict):
        return {}
    return {k: v for k, v in data.items()
            if isinstance(v, dict) and isinstance(v.get("tuning"), dict)}


def store_cache(cache: dict):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def tune_batched(x, y, offsets, degree, interval=None, m_max=None, accum="comp", candidates=None, reps=3,
                 use_cache=True, verbose=False, basis="monomial", stream=None):
    """Best tuning dict for this batch layout (measured by lsefit_plan_autotune,
    or from the cache).

    Returns (tuning, results) where results lists (tuning, ms) per candidate
    measured now (empty when the cache answered)."""
    dev = x.device
    offsets_d = L._to_device(offsets, torch.int64, dev)
    degree_d = L._to_device(degree, torch.int32, dev)
    interval_d = L._to_device(interval, torch.float64, dev) if interval is not None else None
    if m_max is None:
        m_max = int(degree_d.max().item())
    off_host = L._as_host_int64(offsets)
    deg_host = np.ascontiguousarray(
        degree.detach().cpu().numpy() if isinstance(degree, torch.Tensor) else np.asarray(degree), dtype=np.int32)
    S = off_host.size - 1
    key = _device_key(dev, str(x.dtype), str(accum), m_max, layout_signature(off_host), basis)
    with _lock:
        cache = load_cache() if use_cache else {}
        if key in cache:
            return dict(cache[key]["tuning"]), []
    cands = candidates or builtin_candidates()
    n = len(cands)
    arr = (L.Tuning * n)(*[_tuning_struct(c) for c in cands])
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    offp = off_host.ctypes.data_as(ctypes.c_void_p)
    degp = deg_host.ctypes.data_as(ctypes.c_void_p)
    ints = ctypes.c_int64(0)
    wsb = ctypes.c_size_t(0)
    L._check(L.lib.lsefit_plan_autotune_sizes(offp, degp, S, int(m_max), arr, n, sms, ctypes.byref(ints),
                                              ctypes.byref(wsb)), "lsefit_plan_autotune_sizes")
    tasks = torch.empty(max(int(ints.value), 4), dtype=torch.int32, device=dev)
    ws = torch.empty(max(int(wsb.value), 256), dtype=torch.uint8, device=dev)
    X = torch.empty(S, m_max + 1, dtype=torch.float64, device=dev)
    st = torch.empty(S, dtype=torch.int32, device=dev)
    b = L.Batch(x.data_ptr(), y.data_ptr(), offsets_d.data_ptr(), degree_d.data_ptr(),
                interval_d.data_ptr() if interval_d is not None else None, S, int(m_max), L._dtype_code(x),
                L._accum_code(accum), L.BASES[basis])
    best = L.Tuning()
    ms = (ctypes.c_float * n)()
    rc = L.lib.lsefit_plan_autotune(ctypes.byref(b), offp, degp, arr, n, int(reps), L._ptr(tasks), tasks.numel(),
                                    L._ptr(ws), ws.numel(), L._ptr(X), L._ptr(st),
                                    ctypes.c_void_p(L._stream_handle(stream)), ctypes.byref(best), ms)
    L._check(rc, "lsefit_plan_autotune")
    results = [(dict(c), float(ms[i])) for i, c in enumerate(cands)]
    if verbose:
        for c, t in results:
            print(f"  tune {c} -> {t:.3f} ms")
    best_d = _tuning_dict(best)
    best_ms = min(t for _, t in results)
    with _lock:
        cache = load_cache() if use_cache else {}
        cache[key] = {"tuning": best_d, "ms": best_ms, "candidates": [[c, t] for c, t in results]}
        if use_cache:
            store_cache(cache)
    return best_d, results
