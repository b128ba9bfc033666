"""GB300-native screened HSE exact-exchange (HFX) build.

K_{mu nu} = sum_{lambda sigma} (mu lambda | nu sigma)_omega P_{lambda sigma} over Schwarz-
and orbital-cutoff-screened contracted Gaussian shell quartets, evaluated by CUDA
kernels for sm_103a behind the C ABI declared in ``include/hfx.h``.

Importing the package loads nothing; ``paper_2009_03559_gb300.hfx`` loads the CUDA
library and raises if it is missing (there is no CPU path).
"""
__all__ = ["inputs", "hfx"]
