"""GB300-native hot path of the noisy quantum-circuit simulator of
Bogdanov et al., "Numerical and analytical research of the impact of
decoherence on quantum circuits" (arXiv:1412.2293).

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through its C ABI (``include/qs.h``); ``qs`` is the thin ctypes binding.
Importing the package does not load the library: ``inputs`` (seeded
workloads) stays importable on machines without the built library.
"""

__all__ = ["inputs", "qs"]
