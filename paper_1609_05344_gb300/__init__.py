"""GB300-native volumetric-cloud raymarch and TAA resolve (arXiv 1609.05344).

The compute path is libcloudvol.so (CUDA, sm_103a) behind the C ABI in
include/cloudvol.h; ``api`` is its Python binding and ``inputs`` builds the
seeded synthetic workloads.  Importing the package does not load the library;
the first call into ``api`` does, and raises if it has not been built.
"""
__all__ = ["api", "inputs"]
