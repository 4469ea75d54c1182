"""CPU FP64 oracle for the null-space-free (NSF) Maxwell eigensolver.

TEST INFRASTRUCTURE.  This package is the slow, plain reference that the CUDA
library is checked against.  Only the test-suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it; the
library itself never does, and this package never imports the library.

Everything is NumPy / SciPy in complex128, written in the paper's order and
notation (Chern, Hsieh, Huang, Lin, Wang, "Singular value decompositions for
single-curl operators in three-dimensional Maxwell's equations for complex
media"):

* :mod:`oracle.yee`   -- Section 2: the Yee single-curl matrix C (eqs. (mtx_C),
  (mtx_C123), (mtx_K_n1)), the twisted DFT basis T (eq. (mtx_T)), the
  diagonalisation theorem (thm:SchurDecomp_Ci), the Lemma's Lambda_q and
  Lambda_p (eq. (mtx_Lambda_p_q)), the bases Pi_0, Pi_1, Pi_2 (eqs. (mtx_Q0),
  (mtx_Pi_1), (mtx_Pi_2)) and the SVD theorem (thm:svd_C).
* :mod:`oracle.media` -- Section 4.3: chiral and pseudochiral tensors xi_d,
  zeta_d (eqs. (chiral_para_mtx), (pseudo_chiral_para_mtx)) built from a
  :class:`workloads.Medium`.
* :mod:`oracle.gep`   -- Section 3: the discrete GEP (eq. (discrete_GEP_EH)) solved
  directly, densely (tier O1) or by sparse shift-invert (tier O2), through the
  equivalent Hermitian-definite pencil; eigenvalue gradients; the
  Cholesky-scaled Hermitian matrix A of Theorem lem:skew-symm_A (eq. (mtx_A)).
* :mod:`oracle.nfgep` -- Sections 4.1-4.2: the HHPD-NFGEP (thm:NFSEP_real_ew),
  the factored A_r (eq. (factor_mtx)) applied with FFTs (tier O3), B_r, CG
  (eq. (spd_LS)), an ARPACK invert-Lanczos eigensolve, and the fields
  x = [E; H] = B^{-1} diag(P_r, Q_r) y of Algorithm 1's final step; with
  :func:`oracle.gep.gep_residual`, the relative residual of (omega, x) in the
  GEP itself.
* :mod:`oracle.nfsep` -- Section 4 (thm:nfep) and Algorithm 1's second branch:
  the null space free standard eigenproblem (eq. NFSEP_org) for any
  nonsingular B (media outside the Assumption: lossy, non-reciprocal,
  strongly coupled bi-isotropic), shift-and-invert Arnoldi with GMRES, and the
  field recovery of that branch.

Readings of the paper that the oracle fixes (the paper is silent or misprints):

Equations are cited by their LaTeX labels in the paper's source.

* Pi_1 normalisation: the second expression of eq. (mtx_Pi_1) omits a factor
  Lambda_q^{-1}; the oracle divides the printed vector by
  sqrt(Lambda_q * Lambda_p^* Lambda_p), which equals the first (projection)
  expression and makes Q unitary (pinned by the tests).
* mesh length delta_l = a / n_l; alpha = 2, beta = 3 by default (the Lemma
  only needs alpha*delta_x != beta*delta_y and delta_z != beta*delta_y).
* k enters only through k . a_l ("kdota"): the phase over a_l is
  exp(i 2 pi k . a_l).
"""
