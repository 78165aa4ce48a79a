"""GB300-native (sm_103a) parallel orbital-updating (ParO) hot path.

The compute path lives in the C-ABI shared library ``libparo.so`` (CUDA
kernels under ``csrc/``, interface in ``include/paro.h``).  ``binding`` is a
thin ctypes layer with the same entry-point names; ``workloads`` generates the
seeded synthetic inputs.  Importing this package loads nothing: the library is
opened on first use and a missing build raises instead of falling back.
"""
__all__ = ["binding", "workloads"]
