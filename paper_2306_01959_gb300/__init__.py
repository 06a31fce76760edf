"""GB300-native WCSPH particle-interaction pass (sm_103a CUDA behind a C ABI).

Importing the package loads nothing; ``paper_2306_01959_gb300.sph`` loads the
CUDA library ``libsph.so`` and fails loudly when it has not been built.
"""
__all__ = ["workloads", "sph", "build"]
