"""GB300-native FDTD-Bath: Yee FDTD with Lorentz-Bath polarization in hand-written sm_103a CUDA.

Modules:
    fdtdbath  -- Python binding of the C ABI (include/fdtdbath.h); loads the CUDA library.
    workloads -- seeded synthetic problem descriptions (no method arithmetic).
    build     -- in-tree nvcc build of the library.

Importing the package loads nothing; the CUDA library is loaded on first use by
``fdtdbath.lib()`` and there is no CPU fallback.
"""
__all__ = ["fdtdbath", "workloads", "build"]
