"""GB300-native hot path of the relativistic-reference-frame (boosted-frame) PIC method.

The compute path is the C-ABI CUDA library ``libgbpic.so`` (sm_103a kernels) declared
in ``include/gbpic.h``; :mod:`paper_2411_04703_gb300.api` is its thin ctypes binding.
The library is loaded lazily on first use so that the workload definitions in
:mod:`paper_2411_04703_gb300.workloads` import on machines without a GPU.
"""
__all__ = ["api", "workloads"]
