"""GB300-native second-order self-gravity of thin disks on nested grids.

The compute path is the CUDA library ``libsgf.so`` (C ABI declared in
``include/sgf.h``); ``paper_1603_03142_gb300.sgf`` is its thin ctypes binding.
``workloads`` builds seeded synthetic inputs.  Importing the package itself
loads nothing native.
"""
__all__ = ["sgf", "workloads"]
