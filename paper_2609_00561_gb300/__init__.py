"""GB300 block-multicolor ICCG: the CUDA library libiccg.so and its binding.

Importing the package does not load the CUDA library; ``iccg.load()`` (called
by every binding function) does, and raises when it has not been built.
"""
from . import iccg  # noqa: F401

__all__ = ["iccg"]
