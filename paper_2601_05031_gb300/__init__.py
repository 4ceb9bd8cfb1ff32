"""GB300 vorticity--stream-vector phase-field step (Gallen et al.).

The compute path is the CUDA library ``_lib/libvsv.so`` (C ABI in
include/vsv.h); ``vsv`` is its same-name Python binding and ``sim`` a thin
convenience wrapper that owns the torch workspace.  Importing the package
does not load the library; the first call into ``vsv`` does, and fails
loudly when it has not been built.
"""
__all__ = ["vsv", "sim", "build"]
