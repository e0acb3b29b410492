"""FP64 CPU oracle for the HDG trace operator and its nested p/h multigrid.

This package is TEST INFRASTRUCTURE. Only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it. The
GPU library never imports, links or calls anything here, and nothing here
imports the GPU library: the two share no code. Inputs (coefficient fields,
right-hand sides) are passed in as arrays produced by the seeded generators in
``paper_1705_09907_gb300.inputs``, which hold none of the method's arithmetic.

Everything is plain numpy/scipy in float64, written to be checked against the
paper (Fabien, Knepley, Mills, Riviere, "Manycore parallel computing for a
hybridizable discontinuous Galerkin nested multigrid method", arXiv 1705.09907)
by eye: no blocking, fusion or reordering beyond the definitions.

Modules
  quadrature  GL / GLL rules, barycentric Lagrange evaluation (Sec. 4)
  mesh        Cartesian mesh numbering (element / edge / face maps, Alg. 3 maps)
  hdg         local HDG matrices (Eqs. eq_h1-eq_h3, static_1/static_2), local
              solver (Eq. shur0), condensed trace matrix (Eq. shur1), condensed
              right-hand side, recovery, the uncondensed global system, and the
              assembly-free apply (Alg. 3) written per edge
  gmg         p-multigrid transfers (Eqs. eq_mg_pro, eq_mg_res), additive
              Schwarz smoother (Sec. 6.4.2), p=0 -> Q1 transfer (Eq. eq_h_mg_pro),
              Galerkin h-levels, Chebyshev smoothing, coarse direct solve,
              V-cycles (Algs. 1 and 2) and multigrid-preconditioned CG
  adjoint     gradient of J = 1/2 |lambda - lambda_obs|^2 with respect to the
              per-element log-coefficient and the source samples
"""
