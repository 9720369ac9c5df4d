"""Seeded synthetic workloads for the least-squares polynomial fit.

Shared by the test suite and the benchmark, for the oracle and the CUDA
library alike.  Holds no fitting arithmetic: only random draws, the
evaluation of the random "true" polynomials that generate y, and storage
casts.  Every array is reproducible from its seed: large arrays are drawn in
fixed-size chunks, each from its own child of ``SeedSequence(seed)``, so the
result does not depend on the number of threads used to fill it.

Workloads (the paper's data are (x_i, y_i) pairs, Section II; its worked
example is the 6-point Table I; the sizes below are the scaled-up workloads
this library is measured on):
  * ``single_fp64``   n = 100,000 FP64, x ~ U[0, 10],
                      y = 1.5 - 0.8x + 0.3x^2 - 0.02x^3 + N(0, 0.1^2)
  * ``single_large``  n = 2^28 FP32, x ~ U[-1, 1], y = cubic with N(0, 1)
                      coefficients + N(0, 0.01^2)
  * ``ragged_batch``  65,536 series, lengths round(exp(U(ln 16, ln 65536))),
                      degree ~ U{1..5}, x ~ U[a, a+w] with a ~ U(-100, 100),
                      w ~ U(0.1, 50), y = random polynomial in the mapped
                      variable t in [-1, 1] (N(0, 1) coefficients) + noise at
                      1% of that series' signal RMS
  * ``diff_batch``    4,096 series x 4,096 FP32 points, x ~ U[-1, 1],
                      y = random cubic + N(0, 0.05^2), loss weights N(0, 1)
  * ``precision``     n = 2^24, x ~ U[0, 1000], random degree-m polynomial in
                      the mapped variable + N(0, 1e-3 * RMS); FP32 and BF16
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 1 << 22

SEED_SINGLE_FP64 = 1512
SEED_SINGLE_LARGE = 1513
SEED_RAGGED = 1514
SEED_DIFF = 1515
SEED_PRECISION = 1516
SEED_WEIGHTS = 1517

TRUE_SINGLE_FP64 = (1.5, -0.8, 0.3, -0.02)


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _poly(coef, t):
    """Evaluate sum_k coef[k] t^k (data generation only)."""
    acc = np.zeros_like(t, dtype=np.float64)
    for c in reversed(list(coef)):
        acc = acc * t + c
    return acc


def to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (nearest, ties to even); returns uint16 bits."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    nan = np.isnan(np.asarray(a, dtype=np.float32))
    out = rounded.astype(np.uint16)
    out[nan] = 0x7FC0
    return out


def from_bf16_bits(b: np.ndarray) -> np.ndarray:
    """Exact FP32 values of bfloat16 bit patterns."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def single_fp64(n: int = 100_000, seed: int = SEED_SINGLE_FP64):
    """Single FP64 series with the cubic 1.5 - 0.8x + 0.3x^2 - 0.02x^3 plus N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 10.0, n)
    y = _poly(TRUE_SINGLE_FP64, x) + rng.normal(0.0, 0.1, n)
    return {"x": x, "y": y, "true": np.array(TRUE_SINGLE_FP64), "sigma": 0.1}


def single_large(n: int = 1 << 28, m: int = 3, seed: int = SEED_SINGLE_LARGE,
                 noise: float = 0.01, out_x: np.ndarray | None = None,
                 out_y: np.ndarray | None = None, threads: int | None = None):
    """One long FP32 series on [-1, 1]: degree-m polynomial (N(0,1) coefficients) + noise.

    Drawn in chunks of 2^22 points; ``out_x``/``out_y`` may be preallocated
    (e.g. pinned) FP32 buffers of length n."""
    ss = np.random.SeedSequence(seed)
    coef_ss, data_ss = ss.spawn(2)
    coef = np.random.default_rng(coef_ss).normal(0.0, 1.0, m + 1)
    nchunks = (n + CHUNK - 1) // CHUNK
    kids = data_ss.spawn(nchunks)
    x = out_x if out_x is not None else np.empty(n, dtype=np.float32)
    y = out_y if out_y is not None else np.empty(n, dtype=np.float32)
    assert x.dtype == np.float32 and y.dtype == np.float32 and x.size >= n and y.size >= n

    def work(ci):
        lo = ci * CHUNK
        hi = min(n, lo + CHUNK)
        rng = np.random.default_rng(kids[ci])
        xc = rng.uniform(-1.0, 1.0, hi - lo).astype(np.float32)
        yc = _poly(coef, xc.astype(np.float64)) + rng.normal(0.0, noise, hi - lo)
        x[lo:hi] = xc
        y[lo:hi] = yc.astype(np.float32)

    with ThreadPoolExecutor(threads or _threads()) as ex:
        list(ex.map(work, range(nchunks)))
    return {"x": x[:n], "y": y[:n], "true": coef}


def weights(n: int, seed: int = SEED_WEIGHTS, lo: float = 0.1, hi: float = 3.0,
            out: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """Per-point weights w ~ U[lo, hi], FP32, drawn in chunks of 2^22 (``out``
    may be a preallocated FP32 buffer of length n)."""
    nchunks = (n + CHUNK - 1) // CHUNK
    kids = np.random.SeedSequence(seed).spawn(max(nchunks, 1))
    w = out if out is not None else np.empty(n, dtype=np.float32)
    assert w.dtype == np.float32 and w.size >= n

    def work(ci):
        a = ci * CHUNK
        b = min(n, a + CHUNK)
        w[a:b] = np.random.default_rng(kids[ci]).uniform(lo, hi, b - a).astype(np.float32)

    with ThreadPoolExecutor(threads or _threads()) as ex:
        list(ex.map(work, range(nchunks)))
    return w[:n]


def ragged_lengths(num_series: int, lmin: int, lmax: int, rng) -> np.ndarray:
    """Lengths round(exp(U(ln lmin, ln lmax)))."""
    u = rng.uniform(math.log(lmin), math.log(lmax), num_series)
    return np.clip(np.rint(np.exp(u)), lmin, lmax).astype(np.int64)


def ragged_batch(num_series: int = 65536, lmin: int = 16, lmax: int = 65536,
                 mmin: int = 1, mmax: int = 5, seed: int = SEED_RAGGED,
                 a_range=(-100.0, 100.0), w_range=(0.1, 50.0),
                 noise_frac: float = 0.01, lengths: np.ndarray | None = None,
                 threads: int | None = None):
    """Concatenated ragged batch: x, y FP32 [N], offsets int64 [S+1], degree int32 [S],
    interval FP64 [S, 2] (the [a, a+w] each series was drawn on)."""
    ss = np.random.SeedSequence(seed)
    meta_ss, data_ss = ss.spawn(2)
    rng = np.random.default_rng(meta_ss)
    if lengths is None:
        lengths = ragged_lengths(num_series, lmin, lmax, rng)
    else:
        lengths = np.asarray(lengths, dtype=np.int64)
        num_series = lengths.size
    degree = rng.integers(mmin, mmax + 1, num_series).astype(np.int32)
    a = rng.uniform(a_range[0], a_range[1], num_series)
    w = rng.uniform(w_range[0], w_range[1], num_series)
    offsets = np.zeros(num_series + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    N = int(offsets[-1])
    x = np.empty(N, dtype=np.float32)
    y = np.empty(N, dtype=np.float32)
    # group series into chunks of roughly CHUNK points for threaded drawing
    groups = []
    start = 0
    while start < num_series:
        end = start
        pts = 0
        while end < num_series and (pts < CHUNK or end == start):
            pts += int(lengths[end])
            end += 1
        groups.append((start, end))
        start = end
    kids = data_ss.spawn(len(groups))

    def work(gi):
        s0, s1 = groups[gi]
        g = np.random.default_rng(kids[gi])
        for s in range(s0, s1):
            lo, hi = int(offsets[s]), int(offsets[s + 1])
            k = hi - lo
            xs = g.uniform(a[s], a[s] + w[s], k).astype(np.float32)
            coef = g.normal(0.0, 1.0, int(degree[s]) + 1)
            t = (xs.astype(np.float64) - (a[s] + 0.5 * w[s])) * (2.0 / w[s])
            sig = _poly(coef, t)
            rms = math.sqrt(float(np.mean(sig * sig))) if k else 0.0
            ys = sig + g.normal(0.0, noise_frac * rms, k)
            x[lo:hi] = xs
            y[lo:hi] = ys.astype(np.float32)

    with ThreadPoolExecutor(threads or _threads()) as ex:
        list(ex.map(work, range(len(groups))))
    interval = np.stack([a, a + w], axis=1)
    return {"x": x, "y": y, "offsets": offsets, "degree": degree, "interval": interval}


def diff_batch(num_series: int = 4096, n: int = 4096, m: int = 3, seed: int = SEED_DIFF,
               noise: float = 0.05):
    """Uniform batch for the differentiable fit: x, y FP32 [S, n]; loss weights w [S, m+1]."""
    ss = np.random.SeedSequence(seed)
    c_ss, w_ss, d_ss = ss.spawn(3)
    coef = np.random.default_rng(c_ss).normal(0.0, 1.0, (num_series, m + 1))
    w = np.random.default_rng(w_ss).normal(0.0, 1.0, (num_series, m + 1))
    rng = np.random.default_rng(d_ss)
    x = rng.uniform(-1.0, 1.0, (num_series, n)).astype(np.float32)
    x64 = x.astype(np.float64)
    sig = np.zeros_like(x64)
    for k in range(m, -1, -1):
        sig = sig * x64 + coef[:, k:k + 1]
    y = (sig + rng.normal(0.0, noise, (num_series, n))).astype(np.float32)
    return {"x": x, "y": y, "w": w, "true": coef}


def precision(n: int = 1 << 24, m: int = 3, seed: int = SEED_PRECISION, lo: float = 0.0,
              hi: float = 1000.0, noise_rel: float = 1e-3):
    """Unscaled x ~ U[lo, hi]; y = degree-m polynomial of the mapped t + N(0, noise_rel * RMS).

    Returns FP32 x, y and their BF16 roundings (uint16 bit patterns)."""
    ss = np.random.SeedSequence([seed, m])
    c_ss, d_ss = ss.spawn(2)
    coef = np.random.default_rng(c_ss).normal(0.0, 1.0, m + 1)
    rng = np.random.default_rng(d_ss)
    x = rng.uniform(lo, hi, n).astype(np.float32)
    t = (x.astype(np.float64) - 0.5 * (lo + hi)) * (2.0 / (hi - lo))
    sig = _poly(coef, t)
    rms = math.sqrt(float(np.mean(sig * sig)))
    y = (sig + rng.normal(0.0, noise_rel * rms, n)).astype(np.float32)
    return {"x": x, "y": y, "x_bf16": to_bf16_bits(x), "y_bf16": to_bf16_bits(y),
            "true_t": coef, "interval": (lo, hi)}


def small_series(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, m: int = 3,
                 noise: float = 0.01, dtype=np.float32):
    """A short series for parity tests (sizes that span several tiles and a ragged tail)."""
    rng = np.random.default_rng(seed)
    coef = rng.normal(0.0, 1.0, m + 1)
    x = rng.uniform(lo, hi, n)
    t = (x - 0.5 * (lo + hi)) * (2.0 / (hi - lo))
    y = _poly(coef, t) + rng.normal(0.0, noise, n)
    return {"x": x.astype(dtype), "y": y.astype(dtype), "true_t": coef}
