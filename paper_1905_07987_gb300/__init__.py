"""GB300-native ADER-DG time step with a-posteriori FV subcell limiting (arXiv 1905.07987).

The compute path is the C-ABI shared library ``libader.so`` built from ``csrc/`` (hand-written
sm_103a CUDA kernels); ``ader`` is its thin ctypes binding.  ``synth`` holds seeded synthetic
inputs.  Importing the package does not load the library; the first call into ``ader`` does,
and raises if it is missing (there is no CPU fallback).
"""
