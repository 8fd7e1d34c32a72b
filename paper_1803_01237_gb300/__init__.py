"""GB300-native Histogram Sort with Sampling (Harsh, Kale, Solomonik, SPAA'19).

The compute path lives in the CUDA library ``_lib/libhss.so`` built from
``csrc/``; ``hss`` is a thin ctypes binding over its C ABI (``include/hss.h``).
Importing this package loads nothing heavy; ``from paper_1803_01237_gb300
import hss`` loads torch and the library.
"""
__all__ = ["hss", "inputs"]
