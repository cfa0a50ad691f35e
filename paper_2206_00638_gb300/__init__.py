"""GB300-native SBP-SAT FDTD (arXiv 2206.00638): fused CUDA leapfrog kernels behind a C ABI.

The native library is loaded lazily by :mod:`paper_2206_00638_gb300.sbpsat`;
importing the package itself loads no native code.
"""
__all__ = ["sbpsat", "workloads"]
