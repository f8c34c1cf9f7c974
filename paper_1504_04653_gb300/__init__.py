"""GB300-native sampler of SymPix preconditioner blocks.

The compute path lives in the CUDA library ``libsympix.so`` (sources in
``csrc/``, C ABI in ``include/sympix.h``); :mod:`.sympix` is its ctypes
binding and :mod:`.workloads` generates seeded synthetic inputs.
"""
