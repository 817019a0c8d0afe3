"""GB300-native H-BACA: blocked adaptive cross approximation with on-device
entry generation and the hierarchical low-rank merge (arXiv 1901.06101),
as a C-ABI CUDA library (``libhbaca.so``) with a thin Python binding.

``binding`` loads the library (it must have been built; there is no CPU
fallback); ``inputs`` draws the seeded synthetic workloads.
"""
__all__ = ["binding", "inputs"]
