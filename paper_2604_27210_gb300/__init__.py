"""GB300-native batched implied volatility (Black-76 / Black-Scholes / BSM).

The compute path is the CUDA library libfv.so (C ABI in include/fv.h); the
Python binding is the submodule ``paper_2604_27210_gb300.fv`` (import it
explicitly: it needs the built library and PyTorch).
"""
