"""Plain, slow FP64 CPU oracle for the reduced-quadrature Biot discretisation and its
monolithic multigrid / FGMRES solver (Adler, He, Hu, MacLachlan, Ohm, arXiv 2107.04060).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arms of ``bench.py`` may import it.  The product library
(``paper_2107_04060_gb300``) never imports, calls or links anything here, and nothing here
imports the product library; the two share only the seeded input generators of the
``synthetic`` module.

Every routine follows the paper's definitions step by step, in numpy / scipy with FP64:

  mesh.py      structured triangulation and DoF numbering (Appendix A mesh, Sec. 2.3 DoF counts)
  fem.py       element matrices by exact quadrature and global assembly of the
               reduced-quadrature block operator (Sec. 2.1 block form, Sec. 2.3 a^RQ, App. A)
  transfer.py  block interpolation P = diag(P_u, P_w, P_p), divergence-preserving P_u
               (Sec. 3, Eq. block_interp; Sec. 3.1), R = P^T
  smoothers.py additive Vanka on vertex patches (Sec. 3.2.1) and inexact Braess-Sarazin
               with the fixed-stress Schur approximation (Sec. 3.2.2, App. D)
  mg.py        V-cycle with rediscretised coarse operators and a direct coarsest solve (Sec. 3,
               Eq. TG-Operator-Biot; Sec. 5.1), two-grid measured factor rho_N (Sec. 4.3)
  krylov.py    right-preconditioned flexible GMRES (Sec. 5.1)
  manufactured.py  loads and errors for the steady manufactured problem (Sec. 5.1)
  timedep.py   backward-Euler time stepping on a smooth manufactured solution (Sec. 2.1,
               Eqs. discrete1-3)
  lfa.py       two-grid local Fourier analysis (Sec. 4, App. A-D): Vanka, inexact and exact
               BSR, rediscretised or Galerkin coarse symbols
  omega_table.py  the bench's damping by brute-force LFA minimisation (Sec. 4.3), written to
               tests/golden/omega_lfa.json
  adjoint.py   gradients of a pressure misfit through direct solves (checked by central
               differences)
mg.py also holds W-cycles (gamma = 2) and Galerkin coarse operators; smoothers.py exact BSR
(the pressure step of Eq. bsr_p solved with a sparse LU of S).

Parity status of each function is stated in its docstring ("pinned by ..." or
"parity unpinned").
"""

