"""GB300-native image-domain gridding (IDG) hot path.

The compute lives in the CUDA library ``libidg.so`` behind a C ABI
(``include/idg.h``); ``paper_2502_17789_gb300.idg`` is its thin ctypes
binding.  Importing this package does not load the library.
"""
__all__ = ["idg", "synth"]
