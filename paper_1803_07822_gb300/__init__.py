"""GB300-native curved-space lattice Boltzmann hot path (arXiv 1803.07822).

The C ABI is declared in ``include/cslbm.h``; ``_abi`` binds it with ctypes
and ``lattice.CurvedLattice`` wraps one channel.  ``inputs`` generates the
seeded synthetic charts and boundary data the workloads use.
"""
from ._abi import BF16S, FP16S, FP32, FP64, INFLOW, OUTFLOW, PERIODIC, WALL, CslbmError  # noqa: F401


def build(force: bool = False) -> str:
    """Compile libcslbm.so in-tree (nvcc, sm_103a); return its path."""
    from . import buildlib
    return buildlib.build(force=force)
