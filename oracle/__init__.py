"""CPU oracle for data-driven GMRES on 2D FDFD problems (complex128, numpy/scipy).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of what the paper computes, used to check the CUDA library.  Only
the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library shares no code, constant or
helper with it, and the product path never calls it.

Modules
  fdfd   -- the FDFD operator A(eps, omega) of Eq. 1 on a periodic Yee grid with
            stretched-coordinate PML, and the source vector b (Sec. II).
  gmres  -- restarted GMRES (Eq. 2) and data-driven (augmented) GMRES (Eqs. 3-4,
            supplement Eqs. S1-S7), step by step in the paper's notation.
  pca    -- principal components of training fields (Sec. III, "Principal
            component analysis").
  losses -- projection loss (Eq. 5) and residual loss (Eq. 6).

Parity status: every function is pinned by tests under ``tests/`` against
closed forms, textbook special cases or library routines, except the GMRES
iteration *counts*, which depend on rounding and orthogonalisation order
("parity unpinned": reported side by side, not compared).
"""
