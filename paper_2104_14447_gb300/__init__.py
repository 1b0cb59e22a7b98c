"""GB300-native GMLS stencil generation (arXiv 2104.14447, Sec. 2).

The compute path is the CUDA library ``libgmls`` (built from ``csrc/``) behind
the C ABI declared in ``include/gmls.h``; ``gmls`` is its thin ctypes binding.
Importing the package does not load the native library; ``gmls.load()`` does,
and raises if the library has not been built.
"""
__all__ = ["gmls", "inputs"]
