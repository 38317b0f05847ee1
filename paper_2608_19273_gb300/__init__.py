"""GB300-native batched explicit patch update (DSLHyPE hot path).

``paper_2608_19273_gb300.dh`` is the thin ctypes binding of the C-ABI library
``libdh.so`` (CUDA, sm_103a); ``paper_2608_19273_gb300.synth`` builds seeded
synthetic inputs.  Importing the package loads nothing: the library is loaded
(and must exist) on first use of the binding.
"""
__all__ = ["dh", "synth"]
