"""FP64 CPU oracle for the Polarized SARA primal-dual iteration (arXiv:1801.02417).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package: only the tests, the smoke check and the CPU-baseline leg of the
benchmark do. It shares no code with the CUDA library.

It is a plain, slow, direct restatement of the paper:
  measurement.py  data model and measurement operator phi (Section 2.1, Eq. 5.1
                  meas_op) as a direct DFT (no NUFFT), its adjoint, ||phi||^2;
  wavelets.py     SARA dictionary Psi (Section 4.1): Dirac + Daubechies db1..db8,
                  periodic orthonormal Mallat transforms, scaled by 1/3;
  prox.py         projections and proximity operators of Section 4.3
                  (P_U, P_V, P_E1, P_E2, l2 ball, soft threshold);
  primal_dual.py  Algorithm 1 (one iteration, step order as printed),
                  Algorithm 2 (reweighting), NNLS start, stop-rule statistics.
  tv.py           Algorithm 3 (Section 4.4): TV and l1 + TV problems with and
                  without the polarization constraint.

Every function cites the passage it follows. Where the paper is silent or
inconsistent the oracle takes one documented reading (listed in each module).
"""
