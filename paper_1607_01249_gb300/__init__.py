"""GB300-native tensor permute-scale-add (TTC, arXiv 1607.01249, Eq. 1).

The compute path is the C-ABI library ``libttc.so`` (hand-written sm_103a
CUDA); :mod:`.ttc` is its thin ctypes binding.  Importing this package does
not load the library; :func:`ttc.lib` does, and raises if it is missing.
"""
__all__ = ["ttc", "inputs"]
