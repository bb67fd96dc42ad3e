"""GB300-native ParPaRaw: massively parallel parsing of delimiter-separated
raw data (Stehle & Jacobsen) as hand-written sm_103a CUDA behind a C ABI.

The CUDA library (``libparparaw.so``) is built in place by ``build.build()``;
importing this package does not load it, the first Parser does.  There is no
CPU fallback: without the library every parse raises.
"""
from . import formats  # noqa: F401
from ._abi import TYPE_NAMES, status_string  # noqa: F401

__all__ = ["formats", "Parser", "Output", "Result", "ParparawError", "parse_batch", "Batch", "skip_rows",
           "status_string"]


def __getattr__(name):
    if name in ("Parser", "Output", "Result", "ParparawError", "parse_batch", "Batch", "skip_rows"):
        from . import parser as _p

        return getattr(_p, name)
    raise AttributeError(name)
