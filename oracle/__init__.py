"""Plain FP64 CPU oracle of the DNN-MG patch-correction step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or
runs this package: only the test-suite, the smoke check and the CPU-baseline
leg of the benchmark do.  It shares no code with the CUDA path; the two meet
only through the seeded inputs of ``paper_2307_14837_gb300.inputs``.

Every routine is written for a reader to check against the paper by eye:
per-cell loops over 2x2x2 Gauss points, global vectors assembled in cell
order, library primitives (numpy matmul, scipy sparse LU) where a step is a
plain linear-algebra operation.  Floating point is float64 throughout.

Modules
  mesh      refinement of a hexahedral mesh, patch map dof(P, i), valences,
            boundary kinds, geometry features            (Sec. 5.2)
  fem       Q1/Q1 element integrals with local projection stabilisation,
            theta-scheme residual and right-hand side   (Eqs. (5), (6), (8), (9))
  transfer  prolongation P and restriction R = P^T       (Alg. 1)
  mlp       the patch network with skips and folded normalisation (Sec. 4)
  dnnmg     local restriction Q, extension L, one DNN-MG step   (Alg. 1)
  solve     Newton solve of A_h(x) = F on one level      (Sec. 3.4)
  q2        the paper's Q2/Q2 element with one-level local projection,
            its levels and the nested prolongation        (Sec. 3.2, Eqs. (5), (8))

Parity status of each function is stated in its docstring ("pinned by ..."),
with the pins in tests/test_oracle_*.py.
"""
