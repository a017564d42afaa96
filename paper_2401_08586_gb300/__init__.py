"""GB300 (sm_103a) implementation of the FP16 relative-coordinate cell
link-list (RCLL) neighbour search and SPH density sum of arXiv 2401.08586.

The compute path is the C-ABI library ``libsph.so`` (CUDA, built from
``csrc/``); :mod:`.sph` is a thin ctypes binding with the same entry-point
names.  Importing this package does not load the library; the first call
through :mod:`.sph` does, and it raises if the library is missing.
"""
__all__ = ["sph", "workloads"]
