"""GB300-native Mamute hot path: 3-D acoustic propagator, adjoint and imaging.

The compute lives in the C-ABI library ``libmamute.so`` (CUDA, sm_103a); the
modules here only marshal arguments into it.  Importing the package does not
load the library; the first call does, and fails loudly if it is missing.
"""
__all__ = ["synth"]
