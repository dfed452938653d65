"""FP64 CPU oracle for the symmetric Muller-like HSS solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA library.

Modules
-------
kernels   Entries of the row-scaled symmetric Muller-like matrix (Eq. 15 / the
          block form of Sec. 4.1) and of the unscaled baseline matrix (the
          naive Muller-like system of Sec. 6), the one-point corrected diagonal
          and the right-hand side; dense assembly and dense LU solve.
exact     Separation-of-variables solution of the transmission problem (Sec. 2)
          on the unit disk, used as the closed-form pin.
hss       Proxy-method compression with column IDs (Sec. 4.1), the symmetric
          single-ID and the non-symmetric two-ID variants, the multilevel
          compressed-equation factorisation and solve (Sec. 4.2).

Parity status
-------------
Every function is pinned by tests under ``tests/test_oracle_*.py``.  The paper does not
print its one-point correction terms (Sec. 3.1); the diagonal entries follow the readings
derived in ``kernels.py`` and ``pmchwt.py`` and are pinned by mathematics rather than by
printed values: the O(h^3) convergence of the disk solution and of nested node sets on a
non-convex star, the transparent-obstacle identity, and the limits of the off-diagonal
kernels along the curve (D~ = D*~ = -kappa / 4 pi; the constant term of the hypersingular
kernel, kappa^2 / 24 pi plus the parametrisation-speed term).  What stays unpinned is only
whether the paper's own correction weights differ from these beyond what the convergence
orders fix ("parity unpinned" for those constants, which the paper does not give).
"""
