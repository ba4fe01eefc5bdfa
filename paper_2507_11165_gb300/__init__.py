"""GB300-native interpolation predictor / error-bounded quantizer (cuSZ-Hi, arXiv 2507.11165).

The compute path is the C-ABI library built from ``csrc/`` (hand-written CUDA
for sm_103a); :mod:`.hi` is its thin ctypes binding.  Importing this package
loads nothing: the library is opened on first use and a missing library is an
error, never a fallback.
"""
__all__ = ["hi", "fields"]
