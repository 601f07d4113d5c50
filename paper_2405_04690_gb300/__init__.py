"""GB300-native Galactic-Binary likelihood engine (arXiv:2405.04690 hot path).

The compute path is libgbk.so (hand-written sm_103a CUDA kernels behind a C ABI,
declared in include/gbk.h); ``_lib`` is its thin ctypes binding. Importing this package
loads nothing; the library is loaded on first use and its absence is an error.
"""
__all__ = ["_lib", "synth", "build"]
