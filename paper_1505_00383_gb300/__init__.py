"""GB300-native many-path polynomial homotopy tracker (Verschelde & Yu 2015).

The compute path is the CUDA library ``libht.so`` (hand-written sm_103a
kernels behind the C ABI of ``include/ht.h``); ``ht`` is its thin ctypes
binding.  Importing the binding fails loudly when the library is missing:
there is no CPU fallback.
"""
from . import ht  # noqa: F401

__all__ = ["ht"]
