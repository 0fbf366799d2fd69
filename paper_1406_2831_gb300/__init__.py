"""GB300 (sm_103a) recycling BiCGSTAB: Alg. 2 of Ahuja, Benner, de Sturler and
Feng, "Recycling BiCGSTAB with an Application to Parametric Model Order
Reduction", as hand-written CUDA kernels behind a C ABI (librbicgstab.so).

Submodules
----------
build      compile librbicgstab.so in-tree (nvcc, sm_103a)
rbicgstab  ctypes binding: Solver (Alg. 2, blocked and mixed solves, Alg. 1
           primary + dual), harmonic_ritz, error codes
autograd   torch.autograd.Function: gradients through the dual system
inputs     seeded synthetic systems (stencil operators, right-hand sides)

Importing the package loads nothing; ``rbicgstab.lib()`` loads the library
and raises if it has not been built.
"""
