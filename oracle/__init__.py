"""CPU oracle for recycling BiCGSTAB (Ahuja, Benner, de Sturler, Feng).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the method, written from the paper's definitions so that the CUDA path can be
checked against it.  Only the test suite, the package's ``smoke()`` check and
the benchmark's CPU-baseline leg may import it; the solver library never does,
and it shares no code with the CUDA sources.

Contents
--------
shadow     counter-based generator for the random shadow residual r~_{-1}
           (Alg. 2): SplitMix64 from its published definition.
bicgstab   van der Vorst's BiCGSTAB, written separately (the k = 0 baseline).
rbicgstab  Alg. 2 (RBiCGSTAB): BiCGSTAB on the projected operator of Sec. 3
           from the start of eq. (3.5), the biorthogonalisation of C and C~, and the cycle store used by
           the recycle-space update.
recycle    harmonic Ritz extraction for the recycle-space update between
           systems, and the mode-S sequence driver.
rbicg      Alg. 1 (RBiCG): the primary system and its dual together, with a
           two-sided recycle space.
recycle_two_sided
           the two-sided Petrov-Galerkin update from RBiCG cycles (the
           reading of the generator Sec. 6.2 defers to the RBiCG paper).
bicgstab_l BiCGstab(l) (Sleijpen-Fokkema), plain and on the recycling
           projected operator: the breakdown-robust variant (l = 1 is Alg. 2).
adjoint    gradient of L = ||C_out x||^2 with respect to b, the entries of A
           and the parameters of A(p), from one dual solve A^T lam = dL/dx
           with the recycle space's roles swapped.
dense      small dense helpers used by the pins (principal angles).

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant, brute force (dense LU), a published test vector or
a value the paper prints (Table 1), except where a docstring says
"parity unpinned".
"""
