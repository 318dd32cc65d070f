"""GB300-native pairwise-perturbation CP-ALS (arXiv 1811.10573) hot path.

The compute path is the CUDA library ``libcpals.so`` built from ``csrc/``;
``cpals`` is a thin ctypes binding with the C-ABI's names.
"""
