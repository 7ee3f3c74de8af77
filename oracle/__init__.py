"""Plain FP64 CPU oracle for tree-cotree IETI-DP (Mally, Vazquez, Schoeps).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA library never imports, links or calls anything here, and this package never
imports the library: the two share only the seeded problem generator in
``workloads/`` (which holds no arithmetic of the method).

Modules, each citing the passage of the paper it follows:

* ``bspline``   -- B-spline bases and Gauss quadrature (Sec. 2.2, spline spaces).
* ``lattice``   -- global control-mesh numbering of nodes and edges, Dirichlet edges.
* ``assembly``  -- K_i, M_C, j_i of Sec. 2.2 on curved patches (covariant Piola map).
* ``gauge``     -- tree-cotree splitting and the e/p/r DOF classes of Sec. 3.
* ``monolithic``-- the implicit-Euler system of Eq. (11) on the gauged unknowns,
                   solved by a sparse direct solver (the reference answer).
* ``ietidp``    -- the dual-primal reformulation of Sec. 3 (the unnumbered system
                   after Eq. (12)), solved with PCG and a Dirichlet preconditioner.
* ``manufactured`` -- manufactured solutions and error norms (Sec. 4).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except the
preconditioner's iteration counts (Fig. 2e-f values are not in the text), which
are "parity unpinned" for the count only; the preconditioner's algebra is pinned
through the projection and lower-eigenvalue properties.
"""
