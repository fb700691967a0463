"""GB300-native parareal / L1 / sine-Galerkin solver for quasilinear Caputo
subdiffusion (arXiv 2510.11023).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/psl1.h``); ``psl1`` is its thin ctypes binding and ``workloads``
the seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "psl1", "build"]
