"""GB300-native (sm_103a) self-gravitating SPH right-hand side.

The compute path lives in ``csrc/`` (CUDA kernels behind a C ABI, declared in
``include/sphgb.h``) and is reached through :mod:`paper_1807_08116_gb300.native`.
Importing the package loads nothing; the first native call loads
``libsphgb.so`` and raises if it has not been built.
"""
__all__ = ["ics", "native", "sim"]
