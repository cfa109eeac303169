"""GB300-native Strang-split semi-Lagrangian Vlasov solver (arXiv:1206.3229).

``inputs`` holds the seeded workloads; ``vlasov`` is the ctypes binding of the CUDA library
(``libvlasov.so``), imported lazily so that the input generators load without a GPU.
"""
__all__ = ["inputs", "vlasov"]
