"""GB300-native ADMM for convolutional inverse problems (arXiv 2006.08303).

The CUDA library (libcip.so, C ABI in include/cip.h) is loaded lazily by
``paper_2006_08303_gb300.api``; importing this package does not touch the GPU.
"""
__all__ = ["api", "inputs", "build"]
