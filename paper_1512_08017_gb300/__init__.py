"""GB300-native least-squares polynomial fitting (Dasgupta, arXiv 1512.08017).

The package is the Python face of ``liblsefit.so``: CUDA kernels for sm_103a
behind the C ABI of ``include/lsefit.h``.  The first use of any binding name
loads the library and raises ImportError if it is missing (build it with
``__graft_entry__.build()``); ``paper_1512_08017_gb300._build`` itself never
loads it.
"""
import importlib

_BINDING = "paper_1512_08017_gb300.lsefit"


def __getattr__(name):
    if name.startswith("_"):  # private names and submodules such as _build
        raise AttributeError(name)
    mod = importlib.import_module(_BINDING)
    try:
        return getattr(mod, name)
    except AttributeError:
        raise AttributeError(f"module 'paper_1512_08017_gb300' has no attribute {name!r}") from None
