"""GB300-native normalized Lomb-Scargle periodogram engine.

The compute path is the CUDA library ``liblsp.so`` (built from ``csrc/``) behind
the C ABI declared in ``include/lsp.h``; ``paper_1007_1658_gb300.lsp`` is a thin
ctypes binding with the same names.  Importing this package loads nothing: the
library is opened on first use, and a missing build is an error, never a
fallback.
"""
__all__ = ["lsp", "synth"]
