"""GB300-native additive-kernel NFFT fast summation (arXiv 2504.00480).

The compute path is the CUDA library ``libagp.so`` (sources in ``csrc/``, C ABI
in ``include/agp.h``); ``agp`` is its ctypes binding. Importing this package
does not load the library; the first call into ``agp`` does, and raises if the
library has not been built (``paper_2504_00480_gb300.build.build()``).
"""
__all__ = ["agp", "inputs", "build"]
