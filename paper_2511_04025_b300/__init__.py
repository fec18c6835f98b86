"""shl: B300-native periodic elastic homogenisation of charge-parametrised shells.

The compute path lives in the CUDA library ``libshl.so`` (C-ABI declared in
``include/shl.h``); ``paper_2511_04025_b300.shl`` is its thin Python binding.
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["inputs", "shl"]
