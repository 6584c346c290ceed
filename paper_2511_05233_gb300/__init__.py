"""GB300-native matrix-free DG solver for scale-resolved Li-S cathodes (arXiv 2511.05233).

The compute path is the CUDA library ``libdgls.so`` (sm_103a) behind the C ABI of
``include/dgls.h``; ``paper_2511_05233_gb300.dgls`` is its thin ctypes binding.  Importing
the package does not load the library; ``paper_2511_05233_gb300.dgls.lib()`` does, and
raises if it has not been built.
"""
__all__ = ["inputs", "dgls"]
