"""GB300-native two-sided Lanczos sgn(H)b and its gauge-force VJP (arXiv:1604.08057).

Importing the package loads nothing native; ``binding.load()`` loads the CUDA
library and raises if it has not been built.
"""
__all__ = ["inputs", "binding"]
