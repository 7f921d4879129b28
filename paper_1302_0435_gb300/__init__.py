"""GB300-native assignment step of parallel D2-clustering (arXiv 1302.0435).

The compute path lives in the CUDA library libd2.so (csrc/, C-ABI declared
in include/d2.h); `paper_1302_0435_gb300.d2` is the thin ctypes binding with
the same call names.  `synth` holds the seeded input generators.
Importing this package does not load the CUDA library; `d2.load()` does, and
fails loudly if it is missing.
"""
__all__ = ["d2", "synth"]
