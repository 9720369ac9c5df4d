"""Thin Python binding of the CUDA library ``liblsefit.so`` (ctypes).

Argument marshalling only: every step of the fit runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  Importing this module
loads the library and raises ImportError if it has not been built, so no
code path can silently run without it.

The library computes the least-squares polynomial fit of Dasgupta,
arXiv 1512.08017, Section II (normal equations A X = B with the Hankel
matrix of power sums, solved by Gaussian elimination); see
``include/lsefit.h`` for the exact contract of each entry point.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

# ---------------------------------------------------------------------------
# constants (values of include/lsefit.h)
# ---------------------------------------------------------------------------
OK = 0
ERR_INVALID_ARG = 1
ERR_N_TOO_SMALL = 2
ERR_SINGULAR = 3
ERR_NONFINITE = 4
ERR_BAD_INTERVAL = 5
ERR_WORKSPACE = 6
ERR_CUDA = 7
ERR_UNSUPPORTED = 8
ERR_SCRATCH_LIMIT = 9

F64, F32, BF16 = 0, 1, 2
ACCUM = {"naive": 0, "comp": 1, "f64": 2}
ABI_VERSION = 4  # LSEFIT_ABI_VERSION the structures below are laid out for
MAX_DEGREE = 8
MAX_DEGREE_CHEBYSHEV = 16  # Chebyshev basis with FP64 accumulation

# per-fit status names (same vocabulary as the oracle's)
STATUS_NAMES = {OK: "ok", ERR_N_TOO_SMALL: "n_too_small", ERR_SINGULAR: "singular",
                ERR_NONFINITE: "nonfinite", ERR_BAD_INTERVAL: "bad_interval", ERR_INVALID_ARG: "invalid_arg"}

_DTYPES = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}


class LsefitError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {status_string(code)} (code {code})")
        self.code = code


# ---------------------------------------------------------------------------
# ctypes declarations
# ---------------------------------------------------------------------------
class Batch(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("degree", ctypes.c_void_p), ("interval", ctypes.c_void_p),
                ("num_series", ctypes.c_int64), ("m_max", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("accum", ctypes.c_int32), ("basis", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("warp_max_len", ctypes.c_int32), ("chunk_len", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("task_order", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class Plan(ctypes.Structure):
    _fields_ = [("num_series", ctypes.c_int64), ("total_points", ctypes.c_int64),
                ("n_block_tasks", ctypes.c_int32), ("n_warp_tasks", ctypes.c_int32),
                ("n_split_series", ctypes.c_int32), ("m_max", ctypes.c_int32),
                ("tuning", Tuning), ("grid", ctypes.c_int32), ("num_sms", ctypes.c_int32),
                ("block_tasks", ctypes.c_void_p), ("warp_tasks", ctypes.c_void_p),
                ("class_begin", ctypes.c_int32 * (MAX_DEGREE + 2)),
                ("class_points", ctypes.c_int64 * (MAX_DEGREE + 1)), ("warp_task_len", ctypes.c_int64)]


# (name, restype, argtypes) of every symbol include/lsefit.h declares
_VP, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_INT = ctypes.c_int
SIGNATURES = {
    "lsefit_status_string": (ctypes.c_char_p, [_INT]),
    "lsefit_abi_version": (_INT, []),
    "lsefit_powersums_workspace_size": (_SZ, [_INT]),
    "lsefit_powersums": (_INT, [_VP, _VP, _I64, _INT, _INT, _INT, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "lsefit_solve": (_INT, [_VP, _I64, _INT, _INT, _INT, _VP, _VP, _VP, _VP, _VP]),
    "lsefit_solve_cholesky": (_INT, [_VP, _I64, _INT, _INT, _INT, _VP, _VP, _VP, _VP, _VP]),
    "lsefit_fit": (_INT, [_VP, _VP, _I64, _INT, _INT, _INT, _INT, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "lsefit_fit_noalloc_scratch_bytes": (_SZ, []),
    "lsefit_fit_general_workspace_size": (_SZ, [_INT]),
    "lsefit_fit_general": (_INT, [_VP, _VP, _VP, _I64, _INT, _INT, _INT, _INT, _INT, _VP, _VP, _VP, _VP, _VP, _VP,
                                  _VP, _SZ, _VP]),
    "lsefit_fit_noalloc": (_INT, [_VP, _VP, _I64, _INT, _INT, _INT, _INT, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "lsefit_plan_build": (_INT, [_VP, _VP, _I64, _INT, _VP, _INT, _VP, _VP, _I64, _VP, _I64]),
    "lsefit_batched_workspace_size": (_SZ, [_VP]),
    "lsefit_plan_class_blocks": (_INT, [_VP, _INT, _VP]),
    "lsefit_fit_batched": (_INT, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "lsefit_residuals_workspace_size": (_SZ, [_VP]),
    "lsefit_residuals": (_INT, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "lsefit_range_workspace_size": (_SZ, [_VP]),
    "lsefit_range": (_INT, [_VP, _VP, _VP, _VP, _SZ, _VP]),
    "lsefit_autotune_candidates": (_INT, [_VP, _INT]),
    "lsefit_plan_autotune_sizes": (_INT, [_VP, _VP, _I64, _INT, _VP, _INT, _INT, _VP, _VP]),
    "lsefit_plan_autotune": (_INT, [_VP, _VP, _VP, _VP, _INT, _INT, _VP, _I64, _VP, _SZ, _VP, _VP, _VP, _VP, _VP]),
    "lsefit_driver_version": (_INT, []),
    "lsefit_check_reciprocal": (_INT, [_VP, _VP, _I64, _VP]),
    "lsefit_backward_workspace_size": (_SZ, [_VP]),
    "lsefit_backward": (_INT, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
}


def _load():
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(
            f"liblsefit.so not found at {path}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue  # symbols not yet provided are reported by the ABI test
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()
if lib.lsefit_abi_version() != ABI_VERSION:
    raise ImportError(f"liblsefit.so reports ABI version {lib.lsefit_abi_version()}, this binding expects "
                      f"{ABI_VERSION}: rebuild it (python -c 'import __graft_entry__ as g; g.build()')")


def status_string(code: int) -> str:
    return lib.lsefit_status_string(int(code)).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise LsefitError(rc, what)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    try:
        return _DTYPES[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported point dtype {t.dtype} (float64, float32 or bfloat16)") from None


def _accum_code(accum) -> int:
    if isinstance(accum, int):
        return accum
    return ACCUM[accum]


def _device_of(x: torch.Tensor) -> torch.device:
    if x.is_cuda:
        return x.device
    return torch.device("cuda", torch.cuda.current_device())


# ---------------------------------------------------------------------------
# workspaces (zero-filled once; the library leaves them zeroed after each call)
# ---------------------------------------------------------------------------
_ws_lock = threading.Lock()
_ws_cache: dict = {}


def workspace(kind: str, nbytes: int, device: torch.device, stream_handle: int) -> torch.Tensor:
    """A cached zero-filled workspace for (kind, device, stream), at least nbytes."""
    key = (kind, device.index, stream_handle)
    with _ws_lock:
        ws = _ws_cache.get(key)
        if ws is None or ws.numel() < nbytes:
            ws = torch.zeros(max(nbytes, 256), dtype=torch.uint8, device=device)
            _ws_cache[key] = ws
        return ws


def _interval_tensor(interval, device, count=1):
    if interval is None:
        return None
    if isinstance(interval, torch.Tensor):
        t = interval
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise TypeError("interval must be a contiguous CUDA float64 tensor")
        if t.numel() != 2 * count:
            raise ValueError("interval must hold (lo, hi) per fit")
        return t
    return torch.tensor(interval, dtype=torch.float64, device=device).reshape(-1)


# ---------------------------------------------------------------------------
# single series
# ---------------------------------------------------------------------------
def powersums(x: torch.Tensor, y: torch.Tensor, m: int, accum="comp", interval=None, *,
              sums=None, map_out=None, status=None, stream=None):
    """S_0..S_2m, T_0..T_m of one series (lsefit_powersums).

    x, y: 1-D CUDA (or pinned host) tensors of float64/float32/bfloat16.
    interval: None, (lo, hi), or a CUDA float64 tensor of 2.
    Returns (sums [3m+2] float64, map [2] float64, status [1] int32), all on device."""
    if x.dim() != 1 or x.shape != y.shape or x.dtype != y.dtype:
        raise ValueError("x and y must be 1-D tensors of the same shape and dtype")
    if not (x.is_cuda or x.is_pinned()) or not (y.is_cuda or y.is_pinned()):
        raise ValueError("x and y must be CUDA tensors or pinned host tensors")
    if not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous")
    dev = _device_of(x)
    sh = _stream_handle(stream)
    iv = _interval_tensor(interval, dev)
    if sums is None:
        sums = torch.empty(3 * m + 2, dtype=torch.float64, device=dev)
    if map_out is None:
        map_out = torch.empty(2, dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=dev)
    nbytes = lib.lsefit_powersums_workspace_size(m)
    if nbytes == 0:
        raise ValueError(f"degree {m} outside 1..{MAX_DEGREE}")
    ws = workspace("powersums", nbytes, dev, sh)
    rc = lib.lsefit_powersums(_ptr(x), _ptr(y), x.numel(), _dtype_code(x), int(m), _accum_code(accum),
                              _ptr(iv), _ptr(sums), _ptr(map_out), _ptr(status), _ptr(ws),
                              ws.numel(), ctypes.c_void_p(sh))
    _check(rc, "lsefit_powersums")
    return sums, map_out, status


def solve(sums: torch.Tensor, m: int, m_sums: int | None = None, map=None, accum="comp", *, X=None, Xt=None,
          status=None, stream=None, method="gauss"):
    """Gaussian elimination of the normal equations (lsefit_solve).

    sums: [count, 3*m_sums+2] or [3*m_sums+2] float64 CUDA tensor; accum: the
    accumulation the sums were formed with (sets the singularity threshold).
    Returns (X, Xt, status) with X, Xt [count, m+1] (or [m+1])."""
    single = sums.dim() == 1
    S = sums.reshape(1, -1) if single else sums
    if m_sums is None:
        m_sums = (S.shape[1] - 2) // 3
    if S.shape[1] != 3 * m_sums + 2:
        raise ValueError("sums row length does not match m_sums")
    count = S.shape[0]
    dev = S.device
    if X is None:
        X = torch.empty(count, m + 1, dtype=torch.float64, device=dev)
    if Xt is None:
        Xt = torch.empty(count, m + 1, dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(count, dtype=torch.int32, device=dev)
    fn = lib.lsefit_solve if method == "gauss" else lib.lsefit_solve_cholesky
    if method not in ("gauss", "cholesky"):
        raise ValueError("method is 'gauss' or 'cholesky'")
    rc = fn(_ptr(S), count, int(m_sums), int(m), _accum_code(accum), _ptr(map), _ptr(X),
            _ptr(Xt), _ptr(status), ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "lsefit_solve")
    if single:
        return X.reshape(-1), Xt.reshape(-1), status
    return X, Xt, status


def fit(x: torch.Tensor, y: torch.Tensor, m: int, accum="comp", interval=None, stream=None) -> dict:
    """One series: power sums then Gaussian elimination (two launches).  Device tensors out."""
    sums, mp, st0 = powersums(x, y, m, accum, interval, stream=stream)
    X, Xt, st = solve(sums, m, m, mp, accum, stream=stream)
    return {"X": X, "Xt": Xt, "sums": sums, "map": mp, "status": st}


def fit_degrees(x: torch.Tensor, y: torch.Tensor, m: int, m_lo: int = 1, accum="comp", interval=None, *,
                out: dict | None = None, stream=None) -> dict:
    """One series, every degree m_lo..m from one pass, in one launch (lsefit_fit).

    Returns dict(X [m-m_lo+1, m+1], Xt, sums [3m+2], map [2], status [m-m_lo+1])."""
    if x.dim() != 1 or x.shape != y.shape or x.dtype != y.dtype:
        raise ValueError("x and y must be 1-D tensors of the same shape and dtype")
    if not (x.is_cuda or x.is_pinned()) or not (y.is_cuda or y.is_pinned()):
        raise ValueError("x and y must be CUDA tensors or pinned host tensors")
    if not (1 <= m_lo <= m <= MAX_DEGREE):
        raise ValueError(f"need 1 <= m_lo <= m <= {MAX_DEGREE}")
    dev = _device_of(x)
    sh = _stream_handle(stream)
    iv = _interval_tensor(interval, dev)
    k = m - m_lo + 1
    if out is None:
        out = {"X": torch.empty(k, m + 1, dtype=torch.float64, device=dev),
               "Xt": torch.empty(k, m + 1, dtype=torch.float64, device=dev),
               "sums": torch.empty(3 * m + 2, dtype=torch.float64, device=dev),
               "map": torch.empty(2, dtype=torch.float64, device=dev),
               "status": torch.empty(k, dtype=torch.int32, device=dev)}
    ws = workspace("powersums", lib.lsefit_powersums_workspace_size(m), dev, sh)
    rc = lib.lsefit_fit(_ptr(x), _ptr(y), x.numel(), _dtype_code(x), int(m), int(m_lo), _accum_code(accum),
                        _ptr(iv), _ptr(out["X"]), _ptr(out.get("Xt")), _ptr(out.get("sums")),
                        _ptr(out.get("map")), _ptr(out["status"]), _ptr(ws), ws.numel(), ctypes.c_void_p(sh))
    _check(rc, "lsefit_fit")
    return out


BASES = {"monomial": 0, "chebyshev": 1}


def fit_general(x: torch.Tensor, y: torch.Tensor, m: int, w: torch.Tensor | None = None, basis: str = "monomial",
                m_lo: int | None = None, accum="comp", interval=None, *, out: dict | None = None,
                stream=None) -> dict:
    """Weighted and/or Chebyshev-basis fit of one series (lsefit_fit_general):
    minimises sum_i w_i (y_i - f(t_i))^2, f = sum_k Xb[k] phi_k(t), phi_k = t^k
    or T_k(t).  Degrees m_lo..m (default m alone) from one pass.

    Returns dict(X [k, m+1] monomials of x, Xb [k, m+1] basis coefficients,
    sums [3m+2], map [2], status [k]) with k = m - m_lo + 1."""
    if x.dim() != 1 or x.shape != y.shape or x.dtype != y.dtype:
        raise ValueError("x and y must be 1-D tensors of the same shape and dtype")
    if w is not None and (w.shape != x.shape or w.dtype != x.dtype):
        raise ValueError("w must have the shape and dtype of x")
    for t in (x, y) + ((w,) if w is not None else ()):
        if not (t.is_cuda or t.is_pinned()):
            raise ValueError("x, y and w must be CUDA tensors or pinned host tensors")
    if basis not in BASES:
        raise ValueError(f"basis must be one of {sorted(BASES)}")
    m_lo = m if m_lo is None else m_lo
    mmax = MAX_DEGREE_CHEBYSHEV if basis == "chebyshev" else MAX_DEGREE
    if not (1 <= m_lo <= m <= mmax):
        raise ValueError(f"need 1 <= m_lo <= m <= {mmax}")
    dev = _device_of(x)
    sh = _stream_handle(stream)
    iv = _interval_tensor(interval, dev)
    k = m - m_lo + 1
    if out is None:
        out = {"X": torch.empty(k, m + 1, dtype=torch.float64, device=dev),
               "Xb": torch.empty(k, m + 1, dtype=torch.float64, device=dev),
               "sums": torch.empty(3 * m + 2, dtype=torch.float64, device=dev),
               "map": torch.empty(2, dtype=torch.float64, device=dev),
               "status": torch.empty(k, dtype=torch.int32, device=dev)}
    # the general pass and lsefit_fit both leave the workspace's ticket zeroed: one buffer serves both
    ws = workspace("powersums", lib.lsefit_fit_general_workspace_size(m), dev, sh)
    rc = lib.lsefit_fit_general(_ptr(x), _ptr(y), _ptr(w), x.numel(), _dtype_code(x), int(m), int(m_lo),
                                _accum_code(accum), BASES[basis], _ptr(iv), _ptr(out["X"]), _ptr(out.get("Xb")),
                                _ptr(out.get("sums")), _ptr(out.get("map")), _ptr(out["status"]), _ptr(ws),
                                ws.numel(), ctypes.c_void_p(sh))
    _check(rc, "lsefit_fit_general")
    return out


def status_names(status: torch.Tensor):
    return [STATUS_NAMES.get(int(v), f"code{int(v)}") for v in status.reshape(-1).tolist()]


# ---------------------------------------------------------------------------
# batched ragged series
# ---------------------------------------------------------------------------
def _as_host_int64(a):
    if isinstance(a, torch.Tensor):
        a = a.detach().to("cpu", torch.int64).numpy()
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.int64)


class BatchPlan:
    """Schedule of one batch layout (lsefit_plan_build) with its task arrays on the device.

    Built once per layout (offsets) and reused by every fit of that layout,
    including CUDA graph replays."""

    def __init__(self, offsets, m_max: int, tuning: dict | None = None, device=None, degree=None):
        import numpy as np
        off = _as_host_int64(offsets)
        deg = None
        if degree is not None:
            deg = np.ascontiguousarray(
                degree.detach().cpu().numpy() if isinstance(degree, torch.Tensor) else degree, dtype=np.int32)
        degp = deg.ctypes.data_as(ctypes.c_void_p) if deg is not None else None
        S = off.size - 1
        device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        tun = Tuning()
        for k, v in (tuning or {}).items():
            setattr(tun, k, int(v))
        plan = Plan()
        offp = off.ctypes.data_as(ctypes.c_void_p)
        rc = lib.lsefit_plan_build(offp, degp, S, int(m_max), ctypes.byref(tun), sms, ctypes.byref(plan),
                                   None, 0, None, 0)
        if rc not in (OK, ERR_WORKSPACE):
            _check(rc, "lsefit_plan_build")
        nb, nw = plan.n_block_tasks, plan.n_warp_tasks
        bt = np.zeros(max(4 * nb, 4), dtype=np.int32)
        wt = np.zeros(max(4 * nw, 4), dtype=np.int32)
        rc = lib.lsefit_plan_build(offp, degp, S, int(m_max), ctypes.byref(tun), sms, ctypes.byref(plan),
                                   bt.ctypes.data_as(ctypes.c_void_p), nb,
                                   wt.ctypes.data_as(ctypes.c_void_p), nw)
        _check(rc, "lsefit_plan_build")
        self.block_tasks_host = bt[: 4 * nb].reshape(-1, 4)
        self.warp_tasks_host = wt[: 4 * nw].reshape(-1, 4)
        self.block_tasks = torch.from_numpy(bt).to(device)
        self.warp_tasks = torch.from_numpy(wt).to(device)
        plan.block_tasks = self.block_tasks.data_ptr()
        plan.warp_tasks = self.warp_tasks.data_ptr()
        self.plan = plan
        self.num_series = S
        self.m_max = int(m_max)
        self.device = device
        self.workspace_bytes = lib.lsefit_batched_workspace_size(ctypes.byref(plan))

    @property
    def tuning(self) -> dict:
        t = self.plan.tuning
        return {"warp_max_len": t.warp_max_len, "chunk_len": t.chunk_len,
                "block_threads": t.block_threads, "blocks_per_sm": t.blocks_per_sm, "task_order": t.task_order,
                "schedule": t.schedule}


def _to_device(a, dtype, device):
    if isinstance(a, torch.Tensor):
        if a.device != device or a.dtype != dtype:
            a = a.to(device=device, dtype=dtype)
        return a.contiguous()
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dtype)


def fit_batched(x, y, offsets, degree, interval=None, m_max: int | None = None, accum="comp",
                plan: BatchPlan | None = None, out: dict | None = None, stream=None, basis: str = "monomial") -> dict:
    """Fit every series of a ragged batch (lsefit_fit_batched), one persistent launch.

    x, y: 1-D CUDA tensors (float32/bfloat16/float64), all series concatenated.
    offsets: int64 [S+1]; degree: int32 [S]; interval: float64 [S, 2] or None.
    Host arrays are copied to the device.  basis: "monomial" (the paper's fit)
    or "chebyshev" (Xt then holds the Chebyshev coefficients of t).
    Returns dict(X, Xt, sums, map, status, plan)."""
    if basis not in BASES:
        raise ValueError(f"basis must be one of {sorted(BASES)}")
    if not (isinstance(x, torch.Tensor) and x.is_cuda and isinstance(y, torch.Tensor) and y.is_cuda):
        raise ValueError("x and y must be CUDA tensors")
    if x.dim() != 1 or x.shape != y.shape or x.dtype != y.dtype:
        raise ValueError("x and y must be 1-D tensors of the same shape and dtype")
    dev = x.device
    off_d = _to_device(offsets, torch.int64, dev)
    deg_d = _to_device(degree, torch.int32, dev)
    S = off_d.numel() - 1
    if m_max is None:
        m_max = int(deg_d.max().item()) if S > 0 else 1
    if plan is None:
        plan = BatchPlan(offsets if not isinstance(offsets, torch.Tensor) else off_d, m_max, device=dev,
                         degree=degree)
    if plan.num_series != S or plan.m_max != m_max:
        raise ValueError("plan does not match the batch")
    iv = None
    if interval is not None:
        iv = _to_device(interval, torch.float64, dev)
        if iv.numel() != 2 * S:
            raise ValueError("interval must be [S, 2]")
    nc = m_max + 1
    if out is None:
        out = {"X": torch.empty(S, nc, dtype=torch.float64, device=dev),
               "Xt": torch.empty(S, nc, dtype=torch.float64, device=dev),
               "sums": torch.empty(S, 3 * m_max + 2, dtype=torch.float64, device=dev),
               "map": torch.empty(S, 2, dtype=torch.float64, device=dev),
               "status": torch.empty(S, dtype=torch.int32, device=dev)}
    b = Batch(x.data_ptr(), y.data_ptr(), off_d.data_ptr(), deg_d.data_ptr(),
              iv.data_ptr() if iv is not None else None, S, m_max, _dtype_code(x), _accum_code(accum), BASES[basis])
    sh = _stream_handle(stream)
    ws = workspace("batched", plan.workspace_bytes, dev, sh)
    rc = lib.lsefit_fit_batched(ctypes.byref(b), ctypes.byref(plan.plan), _ptr(out["X"]), _ptr(out.get("Xt")),
                                _ptr(out.get("sums")), _ptr(out.get("map")), _ptr(out["status"]),
                                _ptr(ws), ws.numel(), ctypes.c_void_p(sh))
    _check(rc, "lsefit_fit_batched")
    out["plan"] = plan
    out["basis"] = basis
    # keep the device copies alive for asynchronous use
    out["_inputs"] = (off_d, deg_d, iv)
    return out


def residuals_batched(x, y, offsets, degree, fwd: dict, want_r: bool = False, want_vtr: bool = True,
                      interval_given: bool = True, stream=None) -> dict:
    """SSE, V^T r and optionally the residuals of a batched fit (lsefit_residuals).

    fwd is the dict returned by fit_batched (its plan, Xt and map are used)."""
    plan: BatchPlan = fwd["plan"]
    dev = x.device
    off_d = _to_device(offsets, torch.int64, dev)
    deg_d = _to_device(degree, torch.int32, dev)
    S = off_d.numel() - 1
    out = {"sse": torch.empty(S, dtype=torch.float64, device=dev)}
    if want_vtr:
        out["vtr"] = torch.empty(S, plan.m_max + 1, dtype=torch.float64, device=dev)
    if want_r:
        out["r"] = torch.empty(x.shape, dtype=torch.float64 if x.dtype == torch.float64 else torch.float32,
                               device=dev)
    b = Batch(x.data_ptr(), y.data_ptr(), off_d.data_ptr(), deg_d.data_ptr(), None, S, plan.m_max,
              _dtype_code(x), 0, BASES[fwd.get("basis", "monomial")])
    sh = _stream_handle(stream)
    ws = workspace("residuals", lib.lsefit_residuals_workspace_size(ctypes.byref(plan.plan)), dev, sh)
    rc = lib.lsefit_residuals(ctypes.byref(b), ctypes.byref(plan.plan), _ptr(fwd["Xt"]),
                              _ptr(fwd["map"]) if interval_given else None, _ptr(out.get("r")), _ptr(out["sse"]),
                              _ptr(out.get("vtr")), _ptr(ws), ws.numel(), ctypes.c_void_p(sh))
    _check(rc, "lsefit_residuals")
    return out


def range_batched(x, offsets, plan: BatchPlan | None = None, out=None, stream=None):
    """Per-series [min x, max x] (lsefit_range); float64 [S, 2] on the device."""
    dev = x.device
    off_d = _to_device(offsets, torch.int64, dev)
    S = off_d.numel() - 1
    if plan is None:
        plan = BatchPlan(offsets if not isinstance(offsets, torch.Tensor) else off_d, 1, device=dev)
    if out is None:
        out = torch.empty(S, 2, dtype=torch.float64, device=dev)
    b = Batch(x.data_ptr(), None, off_d.data_ptr(), None, None, S, plan.m_max, _dtype_code(x), 0, 0)
    sh = _stream_handle(stream)
    nbytes = lib.lsefit_range_workspace_size(ctypes.byref(plan.plan))
    ws = workspace("range", nbytes, dev, sh)
    rc = lib.lsefit_range(ctypes.byref(b), ctypes.byref(plan.plan), _ptr(out), _ptr(ws), ws.numel(),
                          ctypes.c_void_p(sh))
    _check(rc, "lsefit_range")
    return out


# ---------------------------------------------------------------------------
# adjoint and autograd
# ---------------------------------------------------------------------------
def backward(x, y, offsets, degree, fwd: dict, gX: torch.Tensor, interval_given: bool = True,
             accum="comp", dx=None, dy=None, status=None, stream=None):
    """dL/dx, dL/dy of a batched fit (lsefit_backward) for gX = dL/dX [S, m_max+1].

    fwd is the dict returned by fit_batched (its plan, sums, Xt and map are used)."""
    plan: BatchPlan = fwd["plan"]
    dev = x.device
    off_d = _to_device(offsets, torch.int64, dev)
    deg_d = _to_device(degree, torch.int32, dev)
    S = off_d.numel() - 1
    gX = _to_device(gX, torch.float64, dev)
    out_dtype = torch.float64 if x.dtype == torch.float64 else torch.float32
    if dx is None:
        dx = torch.empty(x.shape, dtype=out_dtype, device=dev)
    if dy is None:
        dy = torch.empty(y.shape, dtype=out_dtype, device=dev)
    if status is None:
        status = torch.empty(S, dtype=torch.int32, device=dev)
    b = Batch(x.data_ptr(), y.data_ptr(), off_d.data_ptr(), deg_d.data_ptr(), None, S, plan.m_max,
              _dtype_code(x), _accum_code(accum), BASES[fwd.get("basis", "monomial")])
    sh = _stream_handle(stream)
    nbytes = lib.lsefit_backward_workspace_size(ctypes.byref(plan.plan))
    ws = workspace("backward", nbytes, dev, sh)
    rc = lib.lsefit_backward(ctypes.byref(b), ctypes.byref(plan.plan), _ptr(fwd["sums"]), _ptr(fwd["Xt"]),
                             _ptr(fwd["map"]) if interval_given else None, _ptr(gX), _ptr(dx), _ptr(dy),
                             _ptr(status), _ptr(ws), ws.numel(), ctypes.c_void_p(sh))
    _check(rc, "lsefit_backward")
    return dx, dy, status


class LseFitFunction(torch.autograd.Function):
    """X = fit(x, y) per series, differentiable in x and y through lsefit_backward."""

    @staticmethod
    def forward(ctx, x, y, offsets, degree, interval, m_max, accum, plan):
        res = fit_batched(x, y, offsets, degree, interval, m_max=m_max, accum=accum, plan=plan)
        ctx.save_for_backward(x, y)
        ctx.fwd = res
        ctx.meta = (offsets, degree, interval is not None, accum)
        ctx.mark_non_differentiable(res["status"])
        return res["X"], res["status"]

    @staticmethod
    def backward(ctx, gX, _gstatus):
        x, y = ctx.saved_tensors
        offsets, degree, has_interval, accum = ctx.meta
        dx, dy, _ = backward(x, y, offsets, degree, ctx.fwd, gX.contiguous(), interval_given=has_interval,
                             accum=accum)
        return dx.to(x.dtype), dy.to(y.dtype), None, None, None, None, None, None


def fit_differentiable(x, y, offsets, degree, interval=None, m_max=None, accum="comp", plan=None):
    """Batched fit whose coefficients X carry gradients to x and y.  Returns (X, status)."""
    if m_max is None:
        m_max = int(_to_device(degree, torch.int32, x.device).max().item())
    if plan is None:
        plan = BatchPlan(offsets, m_max, device=x.device, degree=degree)
    return LseFitFunction.apply(x, y, offsets, degree, interval, m_max, accum, plan)
