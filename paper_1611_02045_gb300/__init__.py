"""GB300-native hot path of PCG_C (Antoine, Levitt, Tang, arXiv:1611.02045).

libgpe.so (CUDA, C ABI in include/gpe.h) is loaded lazily by
paper_1611_02045_gb300.gpe; importing the package loads nothing.
"""
__all__ = ["gpe", "inputs", "build"]
