"""Plain FP64 CPU oracle for the SEM Poisson/Helmholtz operator solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or constants with the CUDA library; both sides receive the
same seeded inputs from ``seeded_inputs`` and nothing else.

It is written for a reader to check against the paper (Jansson et al.,
"Neko: A modern, portable, and scalable framework for high-fidelity
computational fluid dynamics", arXiv 2107.01243) by eye:

* ``gll``       -- GLL nodes, weights and the derivative matrix D (§2, Eq. 7-8)
* ``mesh``      -- structured hexahedral box, GLL-node coordinates, global
                   numbering for the gather matrix Q^T, Dirichlet mask
                   (§2, Eq. 4-5, Eq. 10)
* ``geometry``  -- geometric factors G^e and the lumped mass B (§2, Eq. 9)
* ``operator``  -- matrix-free local stiffness apply w_e = D^T G_e D u_e and
                   the gather-scatter QQ^T (§2, Eq. 9-10; §3.2)
* ``solve``     -- Jacobi-preconditioned CG on the matrix-free operator (§2,
                   last paragraph; §4 velocity solver)
* ``adjoint``   -- the per-point gradient of a loss with respect to a
                   variable diffusion coefficient (structure of Eq. 9)
* ``projection``-- projection onto previous solutions for successive
                   right-hand sides (§4, Table 2)
* ``schwarz``   -- the two-level additive overlapping Schwarz preconditioner:
                   fast-diagonalisation local solves on grown elements and a
                   trilinear coarse level solved by a few CG iterations (§4)
* ``gmres``     -- flexible GMRES(m) with right preconditioning (§4, Table 2)
* ``pipecg``    -- pipelined PCG, one reduction per iteration (§10 outlook)
* ``dense``     -- brute-force dense element matrices and assembly for tiny
                   meshes, from explicit basis gradients (§2, Eq. 3 and Eq. 9)

Arrays of local (unassembled, "L") values have shape (E, p, p, p) indexed
[e, k, j, i] with i fastest, p = N + 1, matching the Fortran
``w(:,:,:,:)`` storage of Listing 1.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants and brute force (``-m "not gpu"``).  No function is
"parity unpinned".
"""
