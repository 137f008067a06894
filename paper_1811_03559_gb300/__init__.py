"""GB300-native recursive SPIKE banded solver (Spring, Polizzi, Sameh, arXiv 1811.03559).

The solver itself lives in the CUDA/C++ library ``libspike.so`` (sources in
``csrc/``, C ABI in ``include/spike.h``); ``spike`` is its thin ctypes binding.
Importing this package does not load the library; ``spike.lib()`` does, and it
raises if the library is missing (there is no CPU fallback).
"""
__all__ = ["spike", "inputs"]
