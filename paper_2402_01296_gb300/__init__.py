"""GB300-native engine for the ciphertext branch of bi-CryptoNets (arXiv 2402.01296).

The compute lives in the native library libbcn.so (C ABI: include/bcn.h,
hand-written sm_103a CUDA plus host C++ for the client side); ``bcn`` is its
thin Python binding.
"""
__all__ = ["bcn"]
