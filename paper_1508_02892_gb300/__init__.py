"""GB300-native kinetic-electron PIC/MCC step of the 1D hybrid scheme (arXiv 1508.02892).

The compute path is the C-ABI library ``libhybrid1d.so`` (hand-written CUDA for
sm_103a, built by ``paper_1508_02892_gb300.build``); ``paper_1508_02892_gb300.hybrid``
is its thin ctypes binding.  ``workloads`` holds the seeded synthetic inputs.
Importing the package loads nothing; the binding loads the library on first use
and raises if it is missing.
"""
__all__ = ["workloads", "hybrid", "build"]
