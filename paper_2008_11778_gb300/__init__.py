"""GB300-native Anderson-accelerated FWI / LSRTM gradient path.

The compute path is the CUDA library ``libaafwi.so`` (C ABI declared in
include/aafwi.h); ``paper_2008_11778_gb300.aafwi`` is its thin ctypes binding.
Importing this package loads nothing; the binding raises if the library is
missing, and there is no CPU fallback.
"""
__all__ = ["aafwi", "synth"]
