"""GB300-native EULBFS explicit time step (arXiv 2507.03366).

The compute path lives in the CUDA library ``libeulbfs.so`` (sources under
``csrc/``, C ABI in ``include/eulbfs.h``); ``eulbfs`` is its thin ctypes
binding and ``workloads`` holds the seeded synthetic problems.
"""
__all__ = ["workloads"]
