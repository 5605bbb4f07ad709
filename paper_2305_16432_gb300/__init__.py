"""GB300-native learned-preconditioner PCG (arXiv 2305.16432 hot path).

The compute path lives in the CUDA library ``libnpcg.so`` (sources in
``csrc/``, C-ABI in ``include/npcg.h``); ``npcg`` is its thin ctypes binding.
``inputs`` holds the seeded synthetic input generators.
"""
__all__ = ["inputs", "npcg"]
