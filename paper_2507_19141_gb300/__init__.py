"""GB300-native DASH 4D-hash deformation path (arXiv 2507.19141, Sec. 4.2-4.3).

The compute lives in ``libdash.so`` (hand-written CUDA for sm_103a behind a C
ABI, declared in ``include/dash.h``); ``dash`` is its thin ctypes binding.
Importing this package does not load the library: ``from
paper_2507_19141_gb300 import dash`` does, and fails loudly if it is missing.
"""
__all__ = ["dash", "synth"]
