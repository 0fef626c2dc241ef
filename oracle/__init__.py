"""Plain FP64 CPU oracle for the inverse fast multipole method (IFMM).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or call anything in this package.  The product path (the C-ABI library under
``paper_1508_01835_gb300``) never routes through it and shares no code with it.

The oracle follows Coulier, Pouransari and Darve, "The inverse fast multipole
method" (arXiv:1508.01835), step by step, with numpy/scipy primitives only
(matmul, LU solve, QR, SVD) and no blocking or fusion beyond what the paper
states.  Module map:

* ``tree``       uniform octree/quadtree, neighbour list N_i and interaction
                 list I_i (Sec. 2.3), colouring used as the elimination order.
* ``kernels``    the kernel functions: 1/r with a diagonal rule, the Gaussian
                 RBF, and the paper's Eq. (K_ij).
* ``chebyshev``  Chebyshev nodes and the interpolation polynomial of the
                 black-box FMM the paper uses for its initial low-rank
                 representation (Sec. 3, ref. fong09a).
* ``h2``         the raw H^2 operators (P2P, P2M/L2P, M2M/L2L, M2L), the FMM
                 matvec, dense assembly of the H^2 matrix A_n for small N, and
                 dense assembly of the extended sparse matrix E (Eq. Ax=b_extended).
* ``h2_ortho``   the same A_n with orthonormal bases (Sec. 3: Chebyshev
                 operators followed by an SVD) and sigma_0 of that extended
                 matrix -- the alternative reading of sigma_0, unused by the
                 default path.
* ``ifmm``       sigma_0(E) by power iteration (Sec. 2.4), weighted initial
                 bases (footnote to Eq. U_j_recomp), level-by-level elimination
                 with fill-in compression and redirection (Algorithms 1-3),
                 merge to the parent (Eqs. y_merge-K_merge), top dense solve,
                 and the substitution phase.
* ``gmres``      non-restarted GMRES with right or left preconditioning
                 (Sec. 3.2, Appendix B) and block GMRES.

Parity status of each function is stated in its module header.
"""
