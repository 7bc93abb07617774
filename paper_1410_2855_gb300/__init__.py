"""GB300-native bounce-map library for high-Fresnel-number microchip laser
resonators (Okulov, "Two-dimensional periodic and quasiperiodic spatial
structures in microchip laser resonator").

The compute path is the C-ABI shared library built from ``csrc/``; the
``rt`` submodule is its thin ctypes binding.  Importing this package loads
nothing: the library is opened on first use of ``rt``.
"""
__all__ = ["rt", "workloads"]
