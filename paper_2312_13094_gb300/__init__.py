"""GB300-native explicit finite-difference acoustic wave propagation.

The compute path lives in ``libfd.so`` (hand-written CUDA for sm_103a behind a
C ABI declared in ``include/fd.h``); ``binding`` marshals arguments to it.
"""
