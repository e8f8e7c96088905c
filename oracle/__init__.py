"""FP64 CPU oracle for preconditioned GMRES on the IRK stage system.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code with the CUDA path; the two
meet only through the seeded inputs of the ``synth`` module.

What it computes (plain, slow, obviously correct; FP64 throughout):

  fem      P1 mass / stiffness / convection assembly and Dirichlet
           elimination (Section 3, the block system Eq. block_coeff_mtx).
  butcher  Radau IIA and Lobatto IIIC tables from their collocation
           definitions (Section 2, Table 1), the LDU factorisation without
           pivoting (Section 4.1) and the preconditioner coefficient matrices
           A~ of Eq. PrecForm (J, GSL, optimised GSL of Eq. GSLopt, DU, LD).
  amg      smoothed-aggregation AMG (the diagonal-block subsolve of
           Section 4.2, one V-cycle each; parameters as read in the design
           notes: the paper names IFISS smoothed aggregation only).
  irk      the Kronecker operator I (x) M + h A (x) F (Section 4), the block
           preconditioner applications of Section 4.2, restarted
           right-preconditioned flexible GMRES, the IRK time step of
           Section 2 and its discrete adjoint.
  dense    dense tools for tiny meshes (condition numbers of Section 4.3,
           spectra, the stability function).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, values printed in the paper, invariants or brute force; none is
"parity unpinned".
"""
