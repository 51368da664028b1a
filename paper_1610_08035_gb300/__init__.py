"""GB300-native exact inference for state-space temporal Gaussian processes
through their block-tridiagonal precision (SpInGP, arXiv 1610.08035).

The compute path is the C-ABI library ``_lib/libspingp.so`` (hand-written
sm_103a CUDA kernels); :mod:`.spingp` is its thin Python binding.  Importing
this package does not load the library; the first call does, and fails
loudly when it is missing.
"""
