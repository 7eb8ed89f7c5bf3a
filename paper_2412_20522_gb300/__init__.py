"""GB300-native masked Gaussian-splatting rasteriser (MaskGaussian, arXiv 2412.20522).

Submodules load lazily: ``scenes`` (seeded inputs) needs no GPU; ``abi`` loads
the CUDA library ``libmaskgs`` and fails loudly when it is missing.
"""
__all__ = ["scenes", "abi", "rasterize"]
