"""GB300-native regularized-Stokeslet filament library (sm_103a).

The compute path is the C-ABI shared library ``libmrs_gb300.so`` built from ``csrc/``;
``paper_2604_12083_gb300.mrs`` is its thin ctypes binding.  Importing this package loads
nothing; the library is loaded on first use and a missing library is an error (there is no
CPU fallback).
"""
__all__ = ["mrs", "workloads"]
