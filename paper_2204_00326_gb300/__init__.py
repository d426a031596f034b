"""GB300-native DAFMM + HODLR hot path for the 2-D Lippmann-Schwinger solver of
Gujjula & Ambikasaran (arXiv 2204.00326).

The compute lives in ``libdafmm.so`` (hand-written CUDA for sm_103a behind the
C-ABI of ``include/dafmm.h``); :mod:`.native` is its ctypes binding and
:class:`DafmmOperator` a small owner of the library handles.  PyTorch is used
for device memory and streams only.
"""
from . import workloads  # noqa: F401


def build(force: bool = False) -> str:
    """Compile libdafmm.so for sm_103a (in-tree) and return its path."""
    from .builder import build as _b

    return _b(force=force)


def __getattr__(name):
    if name == "DafmmOperator":
        from .operator import DafmmOperator

        return DafmmOperator
    raise AttributeError(name)
