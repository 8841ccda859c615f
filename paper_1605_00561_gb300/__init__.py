"""GB300-native multi-level 2-D discrete wavelet transform (libdwt).

The product is the C ABI in ``include/dwt.h`` implemented by
``lib/libdwt.so`` (CUDA kernels for sm_103a); :mod:`.dwt` is its Python
binding and :mod:`.inputs` holds the seeded synthetic workloads.  Nothing is
loaded at import time; ``from paper_1605_00561_gb300 import dwt`` loads the
library on first use and raises if it has not been built.
"""
__version__ = "0.1.0"
