"""GB300-native lattice Wess-Zumino fermion-matrix library (overlap fermions, FFT apply).

The compute path is libwz.so (hand-written CUDA for sm_103a) behind the C ABI
of include/wz.h; ``paper_1005_3276_gb300.binding`` is the ctypes layer over
it.  Importing the binding loads the library and raises if it is missing
(there is no CPU fallback).
"""
