"""GB300-native exact leverage-score sampling from Khatri-Rao products.

The compute path lives in the CUDA library ``libkrpls.so`` (built from
``csrc/`` for sm_103a); ``krpls`` is a thin ctypes binding over its C ABI.
Importing this package does not load the library; ``krpls.lib()`` does, and
raises if it has not been built.
"""
__all__ = ["krpls", "synth"]
