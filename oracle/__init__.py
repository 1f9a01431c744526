"""CPU correctness oracle for the discrete Gabor transform on a nonseparable lattice.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 restatement
of Wiesmeyr, Holighaus and Soendergaard, "Efficient algorithms for discrete
Gabor transforms on a nonseparable lattice" (arXiv 1307.4569).  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import it.  The product path (the CUDA
library and its Python binding) never imports, links or calls anything here,
and this package imports nothing from the product.

Modules
-------
lattice  integer lattice algebra: normal form (Prop. lattNF), minimal length
         (Prop. minsig), constants c,d,p,q (eqs. cd, pq), coset parameters
         (Prop. mwindec), shear parameters (Theorem shearform and its proof,
         eq. modcond), lengths without frequency shear (Prop. noshearlength).
dgt      the transform itself: direct sum of eq. (DGT) (O1), fold + FFT (O2),
         the separable Zak/polyphase factorisation (O3, eq. rect-flops), the
         coset route (eqs. mw_frop / mw_phases) and the shear route
         (Algorithm 1); synthesis as the adjoint of each.
duals    frame operator, canonical dual and tight windows: dense S (eq.
         frameop), Zak-domain Gram blocks (separable and coset), the shear
         dual (Algorithm 2), and the diagonal closed form for short windows.
grads    gradients of sum log(|c|^2 + eps) with respect to a real signal and a
         real window, through the adjoint.

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against brute force, closed forms or invariants (see each docstring).
"""
