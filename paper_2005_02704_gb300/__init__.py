"""GB300-native Lidar surface segmentation (Mukherjee et al., PReMI 2019).

The compute path lives in the CUDA library ``liblsg.so`` (sources in
``csrc/``, ABI in ``include/lsg.h``); ``lsg`` is its ctypes binding and
``serve`` the continuous-batching front end.  Importing this package does not
load the library; ``lsg.load()`` (called by every entry point) builds it
in-tree when needed and raises if it cannot.
"""

__all__ = ["lsg"]
