"""GB300-native GSW-MTP optical-focus-array library (arXiv 2206.12661).

The compute path lives in the CUDA shared library built from ``csrc/``
(``libofa.so``, C ABI in ``include/ofa.h``); ``ofa`` is its thin ctypes
binding.  PyTorch is used only for device memory and streams.
"""
