"""CPU FP64 oracle for one Newton step of the VMS / generalized-alpha
hyper-elastodynamics scheme (Liu & Marsden, arXiv:1809.06350).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or execute it. The product path (the CUDA library and its Python binding)
never calls into it, and it shares no code with that path: the only common
module is ``paper_1809_06350_gb300.inputs`` (seeded input generators, no method
arithmetic).

What it computes, by plain definition, in float64 (numpy; SciPy's sparse LU
as the direct-solve primitive):

* ``constitutive`` -- rho(p), beta(p) from the Gibbs energy (§2, §5.1), the
  deviatoric stress by the paper's route S~ -> P:S~ -> sigma_dev -> P~ (§2).
* ``element``      -- element residuals R_m, R_p on P1 tetrahedra (Appendix A,
  residual formulas), 4-point quadrature.
* ``system``       -- global residual, the consistent tangent blocks A, B, C, D
  as the exact Jacobian of that residual along the kinematically reduced
  directions (§3.3, eq. K_block_decomposition / NR_smaller_eqn_1 and the
  definitions def_matrix_A / def_matrix_D), obtained by complex-step
  differentiation; Dirichlet elimination; the symmetric diagonal scaling
  (§4.1); explicit Schur complement (§4.2); sparse direct solve.
* ``newton``       -- generalized-alpha parameters (§3.2) and the predictor
  multi-corrector Newton step (§3.3), each linear system solved directly.
* ``schur_hat``    -- the explicit sparse S^ = D - C diag(A)^-1 B (§4.2), a
  power-method bound on diag(S^)^-1 S^ and the Chebyshev polynomial
  preconditioner built on S^ (the stand-in for the paper's multigrid on S^).

Parity pins (tests/test_oracle_*.py) tie every function to something other
than itself: closed forms, finite differences, patch and rigid-motion tests,
the homogeneous uniaxial-compression solution, and algebraic identities.
"""
