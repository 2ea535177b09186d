"""GB300-native validity test of linear hexahedra (Johnen, Weill & Remacle, IMR 2017).

The compute path is a C-ABI shared library of hand-written sm_103a CUDA
kernels (``csrc/``, header ``include/hexval.h``); ``hexval`` is its thin
ctypes binding.  ``synth`` holds the seeded synthetic input generators.
"""
