"""GB300 (sm_103a) parabolic FMM for the space-time Galerkin BEM of the heat equation
(arXiv 2106.15911): V_h / K_h matvecs in hand-written CUDA behind a C ABI (include/pfmm.h).

Submodules: ``pfmm`` (ctypes binding of the C ABI), ``build`` (in-tree nvcc build),
``inputs`` (seeded synthetic meshes and data).  Importing the package loads nothing.
"""
