"""GB300-native Hermite-4 block-timestep N-body force path (arXiv:1104.2700).

The compute path is ``libnbody.so`` (hand-written sm_103a CUDA behind a C
ABI, declared in ``include/nbody.h``); ``paper_1104_2700_gb300.nbody`` is the
thin ctypes binding with the same call names.  ``ics`` draws the seeded
synthetic inputs.  Importing the package does not load the CUDA library;
the binding loads it on first use and raises if it is missing.
"""
__all__ = ["ics", "nbody"]
