"""GB300-native (sm_103a) lattice Green's function convolution.

The compute path lives in the CUDA/C++ shared library built from ``csrc/``
(``_build/liblgf.so``) and is reached through the C-ABI declared in
``include/lgf.h``; ``lgf`` is the thin ctypes binding.  Import ``lgf``
explicitly: importing this package does not load the library, so the input
generators stay usable on machines without a GPU.
"""
