"""GB300-native isogeometric Bratu assembly and Newton-Krylov (PetIGA's hot path).

The compute path is the CUDA library libiga.so (include/iga.h); ``iga`` is its
ctypes binding and ``workloads`` the seeded synthetic inputs.
"""
__all__ = ["iga", "workloads", "build"]
