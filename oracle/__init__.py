"""Plain, slow FP64 CPU oracle for DDELM-NN (test infrastructure only).

Only the tests, the entry module's smoke check and the CPU-baseline leg of the
benchmark may import this package.  The CUDA library never links, calls or
reads anything here, and this package imports nothing from the CUDA side: it
takes a problem as plain arrays and recomputes every step of the method from
the paper's equations.

* ``layout``  -- the decomposition: points, Gamma = Pi u Delta numbering, the
  change of variables T (Sec. 3.2) and the modified flux rows A_m (Sec. 3.2).
* ``ddelm``   -- the structured method in the paper's order: D_ab, d_a
  (Sec. 3), S_Pi and its Cholesky factor, application of K~^+ and (K~^+)^T,
  P = A-bar K-bar^+ B-bar (Sec. 3.1), the mixed system Eq. (nn-mixed), CG, and
  the reconstruction Eq. (coarse_sol_2).
* ``dense``   -- brute force for tiny problems: every global matrix of
  Eqs. (ddelm), (intermediate), (coarse), (nn-mixed) formed literally, with
  numpy's pseudo-inverse.
"""
