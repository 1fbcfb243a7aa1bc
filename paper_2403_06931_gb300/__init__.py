"""Batched subsequence DTW (sDTW) on NVIDIA GB300 (sm_103a).

* ``capi``   -- ctypes binding of the C ABI (include/sdtw.h), same names.
* ``sdtw``   -- PyTorch front end: SdtwContext, SdtwFunction, sdtw_cost.
* ``inputs`` -- seeded synthetic workloads (random walks, cuts, int8 codes).
* ``build``  -- compiles libsdtw.so in-tree for sm_103a.

The library has no CPU path: calls need a GB300 and the built library.
"""
__all__ = ["capi", "inputs", "build"]
