"""GB300-native MLSDC-SH: two-level IMEX spectral deferred corrections for the
rotating shallow-water equations with spherical-harmonic transforms.

The compute path is the C-ABI library built from ``csrc/`` (hand-written CUDA
for sm_103a); ``mlsdc`` is its thin ctypes binding.  Importing this package
does not load the library; the first call into ``mlsdc`` does, and raises if
the library has not been built.
"""
