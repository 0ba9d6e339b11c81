"""GB300-native adaptively compressed exchange (ACE) hot path.

The compute path lives in the CUDA shared library ``libace.so`` (built from
``csrc/``) behind a C ABI; ``paper_1601_07159_gb300.ace`` is the thin ctypes
binding. Importing this package does not load the library; importing
``.ace`` does, and raises if it is missing.
"""
__all__ = ["ace", "synth"]
