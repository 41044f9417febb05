"""GB300 (sm_103a) Galerkin integral-equation solver: FFT matrix-vector product,
GMRES and mixed-precision refinement behind the C ABI of include/ie.h.

The CUDA library is built in-tree by ``paper_1512_06126_gb300.build.build()``;
``paper_1512_06126_gb300.ie`` is its ctypes binding.
"""
