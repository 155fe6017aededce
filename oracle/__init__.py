"""FP64 CPU oracle of the DG-SEM FAS multigrid hot path (test infrastructure).

This package is a plain, slow, obviously correct restatement of the method of
"Adaptive multigrid for high-order discontinuous Galerkin methods based on the
full approximation scheme" (Stiller): the SIP discretization (Sec. 2.2,
Eq. (2)), the multilevel FAS formulation and transfer operators (Sec. 3.2-3.3,
Eq. (4)), the weighted additive Schwarz smoother with fast diagonalization
(Sec. 4.3.1, Eqs. (9)-(11), Alg. 5), the SCG method (Alg. 6), the FAS and CS
V-cycles (Algs. 1-2) and the full multigrid startup (Alg. 4), on Dirichlet,
Neumann or periodic meshes.  Everything is float64 numpy.

It is test infrastructure only: the tests, the smoke check and the CPU
baseline leg of the benchmark use it; the product path never imports it and
shares no code with it.  The only shared module is the seeded input generator
(`paper_2608_14123_b300.workloads`), which holds no arithmetic of the method.

Parity status per function is stated in each module header; functions with no
pin independent of themselves say "parity unpinned".
"""
