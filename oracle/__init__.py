"""Plain FP64 CPU oracle of the two-determinant CCSD / DCSD residuals.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the C-ABI library and its Python binding) never
imports, links or calls anything here, and this package imports nothing from
the product path.  The two share only the seeded input generator ``synth``.

What it computes (arXiv 2401.11935, Section II, Eqs. 2-4):
  * ``ccsd``   -- the single-reference spin-orbital CCSD singles/doubles
                  residual <q| exp(-T) H_N exp(T) |Phi_A> for a general
                  (non-diagonal) Fock matrix, written with the textbook
                  Stanton-Gauss intermediates; the energy Delta E_A (Eq. 2);
                  the distinguishable-cluster (DC) modification of the
                  doubles (Section II applies DC to the doubles as in
                  single-reference DCSD).
  * ``twod``   -- the two-determinant layer: the coefficients
                  c_q = <A_q| exp(T_B) |Phi_B> by cluster-to-CI algebra, the
                  coupling W (the residual element of the A->B double),
                  R1 = R^CC - W c1, R2 = R^CC - W (c2 - A(ij;ab)[t1 c1]),
                  masking of the A->B element (Eqs. 3-4 and the text after
                  them).
  * ``element`` -- single residual elements of the same definitions for
                  systems of any size (DF integrals contracted on demand);
                  pinned element by element against ``twod`` on small
                  systems.
  * ``solve``  -- Jacobi + DIIS iterations and the 2x2 effective Hamiltonian
                  (singlet Delta E_A + W, triplet Delta E_A - W).
  * ``brute``  -- determinant-space brute force (CI vectors, full CI,
                  <S^2>) used only to pin the above.

Parity status: every function is pinned by tests under ``tests/`` except the
DC modification term set, which is "parity unpinned" (the term list of the DC
approximation is defined in the paper's cited DC literature, not in the
paper; pinned here: its switch-off limit, symmetry and invariance, its
closed-shell statement, the two-electron limit and the particle-hole
relabeling, which fixes the balance of its hole and particle terms).
"""
