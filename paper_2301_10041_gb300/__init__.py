"""GB300-native library for the per-step saddle-point solve of the
distributed-Lagrange-multiplier fictitious-domain FSI method
(Boffi, Credali, Gastaldi, Scacchi, arXiv:2301.10041).

The compute path is the CUDA library ``_lib/libfsi_gb300.so`` (C ABI in
``include/fsi.h``); ``paper_2301_10041_gb300.fsi`` is its ctypes binding and
``paper_2301_10041_gb300.build`` compiles it in place.
"""
__all__ = ["fsi", "build"]
