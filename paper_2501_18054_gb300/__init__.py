"""GB300-native PNGF direct-binary-search hot path (arXiv 2501.18054).

``pngf``       ctypes binding of the C ABI (include/pngf.h) and ``DbsContext``
``workloads``  seeded synthetic inputs (FDFD / closed-form Green functions)
``build``      nvcc build of the in-tree shared libraries
"""
__all__ = ["pngf", "workloads", "build"]
