"""GB300 projective-dynamics hot path (arXiv 2405.12484, Sec. 7).

The CUDA library libpdgb300.so (built in-tree by ``build.build()``) holds
every kernel; ``sim`` wraps its C ABI for torch tensors.
"""
__all__ = ["build", "sim"]
