"""GB300-native separable dictionary learning (2D-OMP + Tensor-MOD updates).

Importing the package loads nothing; the CUDA library is opened on first use
by :mod:`paper_2007_03800_gb300.sdl`, which raises if it has not been built.
"""
__all__ = ["sdl", "synth"]
