"""GB300 hierarchical interpolative factorization (HIF) of the 3D seven-point operator.

The compute path is the CUDA library ``libhif.so`` (C ABI in ``include/hif.h``);
``hif`` is its Python binding and ``inputs`` draws the seeded synthetic inputs.
Importing the package does not load the library; the first call does.
"""
__all__ = ["hif", "inputs", "build"]
