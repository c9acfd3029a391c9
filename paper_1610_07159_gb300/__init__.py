"""GB300-native halfway-domain scene-flow solver (Thies et al., arXiv 1610.07159).

The solver itself lives in the CUDA library under ``csrc/`` behind the C ABI
declared in ``include/sf.h``; ``sf`` is its thin ctypes binding. ``scenes``
holds the seeded synthetic input generators.
"""
