"""Gradient-optimised NEP training on one sm_103a GPU.

The compute path is libgnep (CUDA kernels behind the C ABI in include/gnep.h),
reached through ``gnep`` (torch tensors for memory and streams).  ``synth``
draws seeded synthetic structures.  Importing the package does not load the
CUDA library; ``gnep`` loads it on first use and fails loudly if it is absent.
"""
__all__ = ["synth", "gnep", "build"]
