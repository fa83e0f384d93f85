"""GB300-native MOMFBD hot path: wavefront-parameterised loss, Wiener object
and gradient (arXiv:2505.10639, Sec. 2.2.1 and 3.1) as sm_103a CUDA kernels
behind a C ABI (``include/mfbd.h``); this package is the thin Python binding.
"""
