"""The C-ABI library builds, loads without a GPU and exports every declared symbol.

Only host-side behaviour is exercised here (no kernel launches).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsefit.h")


@pytest.fixture(scope="module")
def L():
    from paper_1512_08017_gb300 import _build
    _build.build()
    import paper_1512_08017_gb300 as lib
    return lib


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsefit_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("lsefit_powersums", "lsefit_solve", "lsefit_fit_batched", "lsefit_backward"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    raw = ctypes.CDLL(L.lib._name)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing
    # and the binding declares a signature for each
    assert not [n for n in declared_functions() if n not in L.SIGNATURES]


def test_host_only_calls(L):
    assert L.lib.lsefit_abi_version() == L.ABI_VERSION == 4
    assert L.status_string(L.OK) == "ok"
    assert "singular" in L.status_string(L.ERR_SINGULAR)
    for m in range(1, 9):
        ws = L.lib.lsefit_powersums_workspace_size(m)
        assert ws >= 256 + 8 * (3 * m + 1) and ws % 256 == 0
    assert L.lib.lsefit_powersums_workspace_size(0) == 0
    assert L.lib.lsefit_powersums_workspace_size(9) == 0


def test_argument_errors_before_any_cuda_call(L):
    lib = L.lib
    sums = (ctypes.c_double * 32)()
    # degree out of range, negative n, bad dtype/accum, missing workspace
    assert lib.lsefit_powersums(None, None, 10, L.F32, 0, 1, None, sums, None, None, None, 0, None) == L.ERR_INVALID_ARG
    assert lib.lsefit_powersums(None, None, 10, L.F32, 9, 1, None, sums, None, None, None, 0, None) == L.ERR_INVALID_ARG
    assert lib.lsefit_powersums(None, None, -1, L.F32, 2, 1, None, sums, None, None, None, 0, None) == L.ERR_INVALID_ARG
    assert lib.lsefit_powersums(None, None, 10, 7, 2, 1, None, sums, None, None, None, 0, None) == L.ERR_INVALID_ARG
    assert lib.lsefit_powersums(None, None, 10, L.F32, 2, 5, None, sums, None, None, None, 0, None) == L.ERR_INVALID_ARG
    assert lib.lsefit_powersums(None, None, 10, L.F64, 2, 1, None, sums, None, None, None, 0, None) == L.ERR_UNSUPPORTED
    assert lib.lsefit_powersums(None, None, 10, L.F32, 2, 1, None, sums, None, None, None, 0, None) == L.ERR_INVALID_ARG
    ws = (ctypes.c_ubyte * 512)()
    assert lib.lsefit_powersums(None, None, 0, L.F32, 2, 1, None, sums, None, None, ws, 0, None) == L.ERR_WORKSPACE
    # solve: nothing to do for count 0; degree checks
    X = (ctypes.c_double * 16)()
    assert lib.lsefit_solve(sums, 0, 3, 3, 1, None, X, None, None, None) == L.OK
    assert lib.lsefit_solve(sums, 1, 2, 3, 1, None, X, None, None, None) == L.ERR_INVALID_ARG
    assert lib.lsefit_solve(sums, 1, 9, 3, 1, None, X, None, None, None) == L.ERR_INVALID_ARG
    assert lib.lsefit_solve(sums, -1, 3, 3, 1, None, X, None, None, None) == L.ERR_INVALID_ARG
    assert lib.lsefit_solve(sums, 1, 3, 3, 7, None, X, None, None, None) == L.ERR_INVALID_ARG
