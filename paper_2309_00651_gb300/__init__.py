"""Gamma-point Hartree-Fock exact exchange (E_x and V_x phi) on GB300.

The CUDA library ``libhfx`` (built from ``csrc/``) does all of the work; ``hfx`` is
its ctypes binding and ``inputs`` builds seeded synthetic workloads.
"""
__all__ = ["inputs", "hfx"]
