"""GB300-native Maxwell–Bloch FDTD step of the 3D+1 random-laser model.

The hot path (H pass, fused E / gain / noise / population pass, probes,
batched ensemble, reverse-time adjoint) runs in hand-written sm_103a CUDA in
``libmbfdtd.so`` behind the C ABI of ``include/mb_fdtd.h``; ``binding`` is its
ctypes binding and ``inputs`` the seeded input generators.
"""
from .binding import MBSimulation, MBError, MBLibraryError, load_library, mb_default_params  # noqa: F401

__all__ = ["MBSimulation", "MBError", "MBLibraryError", "load_library", "mb_default_params"]
