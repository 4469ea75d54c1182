/*
 * nfs.h -- C ABI of libnfs: the null-space-free (NSF) eigensolver hot path for
 * the discrete 3-D Maxwell equations in chiral and pseudochiral media, on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Chern, Hsieh, Huang, Lin, Wang, "Singular value decompositions for
 * single-curl operators in three-dimensional Maxwell's equations for complex
 * media".  Equations are cited by their labels in the paper's source.
 *
 *   C = P_r Sigma_r Q_r^*            SVD of the Yee single-curl operator (thm:svd_C)
 *   B_r y = omega^{-1} A_r y         HHPD-NFGEP (thm:NFSEP_real_ew, eq. NFSEP_spd_1)
 *   A_r   = diag(P_r^*, Q_r^*) M diag(P_r, Q_r)         eq. (factor_mtx)
 *
 * Vector layout (every 4n-vector crossing this ABI):
 *   u = [u1a | u1b | u2a | u2b], each block n = n1*n2*n3 complex numbers in
 *   spectral order (i3, i2, i1), i1 fastest.  u1a, u1b are the coefficients of
 *   the columns P_2, P_1 of P_r; u2a, u2b those of Q_1, Q_2 of Q_r.  Complex
 *   numbers are interleaved (re, im): double2 for NFS_C128, float2 for NFS_C64.
 *
 * Material layout: per-component real arrays [3][n3][n2][n1], x fastest,
 * component c sampled at its own Yee edge location by the caller (the library
 * does no averaging; the paper, end of Section 3, leaves that stencil open).
 *
 * Ownership: a context copies everything it needs from the caller at setup
 * and owns all device workspaces; vector arguments are caller-owned DEVICE
 * pointers, used on the context's stream, never retained after a call
 * returns.  No call allocates device memory except nfs_setup, nfs_setup_batch
 * and the first nfs_eigs / nfs_eigs_batch with a larger basis than any before.
 *
 * Errors: every int-returning call returns NFS_OK (0) or a negative NFS_E*
 * code; no C++ exception crosses the ABI.  nfs_strerror gives a message.
 * Calls on one context are not thread-safe.
 */
#ifndef NFS_H
#define NFS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes -------------------------------------------------------- */
#define NFS_OK            0
#define NFS_EINVAL       (-1)   /* bad pointer, size, option or enum             */
#define NFS_EUNSUPPORTED (-2)   /* non-orthogonal lattice, n1 != n2, or a grid   */
                                /* size not one of 8,12,16,24,32,48,64,96,128    */
#define NFS_EKPOINT      (-3)   /* every k.a_l integer: Lambda_q singular (Lemma) */
#define NFS_EBASIS       (-4)   /* alpha, beta violate the Lemma: Lambda_p = 0    */
#define NFS_ENOTHPD      (-5)   /* mu <= 0 or Phi <= 0: Assumption (eq. assump)   */
#define NFS_ENOCONV      (-6)   /* iteration limit reached (info still filled)    */
#define NFS_EBREAKDOWN   (-7)   /* CG p^*Ap <= 0 or NaN; Lanczos lost rank        */
#define NFS_ETIMEOUT     (-8)   /* a bounded device-side wait gave up             */
#define NFS_ECUDA        (-9)   /* a CUDA runtime error                          */
#define NFS_ENOMEM       (-10)  /* device allocation failed                      */

/* ---- enums --------------------------------------------------------------- */
#define NFS_MEDIUM_CHIRAL       0  /* xi_d = i gamma, zeta_d = -i gamma, per component   */
#define NFS_MEDIUM_PSEUDOCHIRAL 1  /* xi_d = i gamma on the (axis_a, axis_b) pair only   */

#define NFS_PREC_FP64  0  /* complex128 matvec, CG and Lanczos                    */
#define NFS_PREC_MIXED 1  /* complex64 matvec + CG; refinement residuals with the
                           * double-single product; FP64 Lanczos                 */

#define NFS_C128 0        /* vector element type: double2                         */
#define NFS_C64  1        /* vector element type: float2                          */
#define NFS_C128_DS 2     /* double2 vectors, product in double-single arithmetic
                           * (float pairs, ~1e-14; mixed contexts, nfs_matvec only) */

typedef struct nfs_ctx nfs_ctx;

/* Section 4.3, eqs. (chiral_para_mtx) and (pseudo_chiral_para_mtx), with a
 * diagonal permittivity and permeability.  All pointers are HOST pointers and
 * are copied by nfs_setup. */
typedef struct {
  int kind;              /* NFS_MEDIUM_*                                          */
  int axis_a, axis_b;    /* pseudochiral coupled pair (0 = x, 1 = y, 2 = z), a!=b */
  const double* eps;     /* [3][n3][n2][n1], > 0                                  */
  const double* mu;      /* [3][n3][n2][n1], > 0, or NULL meaning mu = 1          */
  const double* gamma;   /* chiral: [3][n3][n2][n1]; pseudochiral: [n3][n2][n1]   */
} nfs_material;

typedef struct {
  int precision;           /* NFS_PREC_FP64 or NFS_PREC_MIXED                     */
  double alpha, beta;      /* free parameters of Lambda_p (eq. mtx_Lambda_p_q)    */
  double cg_tol;           /* relative residual ||b - A_r x|| / ||b|| to reach    */
  int cg_maxit;            /* CG iteration cap (per refinement step when mixed)   */
  double inner_tol;        /* mixed: residual reduction of each FP32 inner solve
                            * (looser when the remaining reduction to cg_tol is
                            * smaller)                                          */
  int max_refine;          /* mixed: cap on FP64 refinement steps                 */
  double eig_tol;          /* Lanczos: Ritz residual <= eig_tol * |theta|         */
  int ncv;                 /* Lanczos basis size; > 0: fixed, and the basis is
                            * allocated by nfs_setup; 0: max(3 nev, 2 nev + 2,
                            * min(12 nev, 320)) (no restart for most solves)   */
  int max_restarts;        /* thick-restart cap                                   */
  double orth_tol;         /* Lanczos semi-orthogonality level: when the measured
                            * loss of A_r-orthogonality of a new vector to the
                            * older basis exceeds it, those components are
                            * removed; 0 = every step.  Default 1e-10            */
  int deflation_checks;    /* Lanczos: after convergence, up to this many checks
                            * for eigenvalues a single start vector misses (the
                            * further copies of a degenerate one): lock the nev
                            * Ritz vectors, restart from a random vector
                            * A_r-orthogonal to them and converge the next
                            * eigenvalue; a check that finds one among the nev
                            * smallest takes it in and is followed by another.
                            * 0 (default, the paper's procedure) = none; 0..16 */
  unsigned long long seed; /* starting-vector seed                                */
  void* stream;            /* cudaStream_t for every launch; NULL = default       */
} nfs_options;

typedef struct {
  int iterations;          /* total CG iterations (inner FP32 ones when mixed)    */
  int refinements;         /* FP64 residual refinements (mixed), else 0           */
  double rel_residual;     /* final ||b - A_r x|| / ||b||, FP64                   */
  int status;              /* NFS_OK, NFS_ENOCONV or NFS_EBREAKDOWN               */
} nfs_solve_info;

typedef struct {
  int lanczos_steps;       /* operator applications (one CG solve each)           */
  int restarts;
  long long cg_iterations; /* summed over every solve                             */
  long long matvecs_c64;
  long long matvecs_c128;
  int nconv;               /* wanted Ritz pairs that met eig_tol                   */
  double max_ritz_residual;/* max over returned pairs of |beta y_m| / |theta|      */
  int status;
  long long kernel_launches; /* kernels the library launched during the call (CUDA
                              * graph nodes included); in a batch, those of the
                              * problem's whole class                                */
  /* host wall-clock split of the call (the class's, in a batch): total; inside
   * the CG iteration loops; the rest of the linear solves (residual
   * refinement); host projected eigensolves; then the Lanczos phases. */
  double seconds_total;
  double seconds_cg;
  double seconds_refine;
  double seconds_ritz;
  double seconds_recurrence; /* three-term recurrence (FP64)                       */
  double seconds_orth;       /* orthogonality monitor and re-orthogonalisation     */
  double seconds_vectors;    /* forming the returned Ritz vectors                  */
  int reorthogonalisations;  /* steps that re-orthogonalised                       */
  int deflation_checks;      /* deflation checks run (opt.deflation_checks)        */
} nfs_eigs_info;

/* Defaults: FP64, alpha = 2, beta = 3, cg_tol 1e-12, cg_maxit 2000,
 * inner_tol 1e-6, max_refine 8, eig_tol 1e-10, ncv 0, max_restarts 200,
 * orth_tol 1e-10, deflation_checks 0, seed 1, default stream. */
void nfs_default_options(nfs_options* opt);

/* Build a context for one Bloch problem (Algorithm alg:NullSpaceFree, steps
 * 1-3: the Lambda tables, Lambda_q, Lambda_p; Pi_1, Pi_2 are evaluated on the
 * fly from them).
 *   grid[3]   = (n1, n2, n3), each in {8,12,16,24,32,48,64,96,128}, n1 = n2
 *   lattice   = 9 doubles, row l = a_l; must be diagonal (orthorhombic).
 *               NULL means the unit cube (a = 1).
 *   k[3]      = Bloch vector divided by 2 pi (Cartesian); the phase across a_l
 *               is exp(i 2 pi k.a_l) (eq. quasi_periodic).
 *   mat, opt  = copied; opt may be NULL (defaults).
 * Checks the Lemma (lem:nonsingular_full_rank) -> NFS_EKPOINT / NFS_EBASIS and
 * the Assumption (eq. assump) -> NFS_ENOTHPD.  On error *out is NULL. */
int nfs_setup(nfs_ctx** out, const int grid[3], const double* lattice, const double k[3],
              const nfs_material* mat, const nfs_options* opt);

/* Au = A_r u (eq. factor_mtx / eq. spd_LS) in the given element type.  u and
 * Au are device pointers to 4n complex numbers and must not overlap.
 * NFS_C128_DS: complex128 vectors, product in double-single arithmetic (~1e-14;
 * MIXED contexts only, else NFS_EINVAL); it uses the context's CG workspace,
 * so it must not overlap an nfs_cg_solve or nfs_eigs on the same context. */
int nfs_matvec(nfs_ctx* ctx, int dtype, const void* u, void* Au);

/* Run only the passes of nfs_matvec selected by `mask` (bit 0: pass 1,
 * spectral assembly + inverse DFT along x, y; bit 1: pass 2, inverse DFT
 * along z + material product + forward DFT along z; bit 2: pass 3, forward
 * DFT along y, x + projection onto P_r^*, Q_r^*; where the xy plane does not
 * fit in shared memory -- complex128 at 128 -- passes 1 and 3 are two kernels
 * each).  Passes communicate through the context's field workspace, so mask 7
 * equals nfs_matvec; other masks exist to time the passes one by one.  Same
 * arguments as nfs_matvec (NFS_C128 and NFS_C64 only). */
int nfs_matvec_passes(nfs_ctx* ctx, int dtype, int mask, const void* u, void* Au);

/* out = B_r v = i [Sigma_r^{-1} v2; -Sigma_r^{-1} v1] (eq. NFSEP_spd_1), with
 * v1 = [v1a; v1b], v2 = [v2a; v2b]; device complex128, 4n each. */
int nfs_apply_Br(nfs_ctx* ctx, const void* v, void* out);

/* Solve A_r x = b by unpreconditioned CG (Section 4.2).  b, x: device
 * complex128 (4n); x holds the initial guess on entry.  FP64 contexts run CG
 * in complex128; MIXED contexts run complex64 CG inside iterative refinement
 * whose residuals b - A_r x come from the double-single product, or, once the
 * residual is below 2.5e4 cg_tol |b|, from the complex64 product of the small
 * correction.  info may be NULL. */
int nfs_cg_solve(nfs_ctx* ctx, const void* b, void* x, nfs_solve_info* info);

/* The nev smallest positive eigenvalues omega of the GEP (eq.
 * discrete_GEP_EH), by thick-restart invert Lanczos on the HHPD-NFGEP: the
 * nev largest theta = 1/omega of B_r y = theta A_r y.  The basis is FP64 and
 * A_r-orthogonal: FP64 three-term recurrence, and every step the inner
 * products with all older vectors in double-single arithmetic, removing them
 * when they exceed opt.orth_tol.  A single start vector finds one copy of an
 * exactly degenerate eigenvalue (symmetric media and k-points); with
 * opt.deflation_checks > 0 the converged pairs are locked and the search
 * restarted from a random vector A_r-orthogonal to them, which brings in the
 * missing copies.  omega: HOST array of nev doubles, ascending.
 * Y: device complex128 array [nev][4n] of A_r-normalised eigenvectors y, or
 * NULL.  info may be NULL.  Returns NFS_ENOCONV (results still written) if the
 * restart cap is hit first. */
int nfs_eigs(nfs_ctx* ctx, int nev, double* omega, void* Y, nfs_eigs_info* info);

/* Residuals of eigenpairs of the HHPD-NFGEP B_r y = omega^{-1} A_r y
 * (thm:NFSEP_real_ew; eq. NFSEP_spd_1 for B_r):
 *   res[j] = || A_r y_j - omega_j B_r y_j ||_2 / || y_j ||_2   (scale-free),
 * with the complex128 product and B_r on the device, FP64 sums.
 *   omega: HOST, m doubles.  Y: DEVICE complex128 [m][4n] (as nfs_eigs
 *   writes it).  res: HOST, m doubles.
 * Synchronises the context's work stream.  Single-problem contexts only. */
int nfs_residuals(nfs_ctx* ctx, int m, const double* omega, const void* Y, double* res);

/* Allocate now the device memory an nfs_eigs(ctx, nev, ...) call uses (the
 * Lanczos basis of opt.ncv, or of the default size for nev, its shadows, the
 * reduction scratch and the restart rotation matrix), so that the eigensolve
 * itself allocates nothing.  Contexts set up with opt.ncv > 0 have it already.
 * The default size depends on nev only, never on the free device memory:
 * NFS_ENOMEM when it does not fit (choose a smaller opt.ncv, e.g. the paper's
 * 3 nev).  A later nfs_eigs with a larger basis reallocates.  On a context of
 * nfs_setup_biiso it reserves what nfs_nfsep_eigs(ctx, nev, ...) uses instead:
 * the Arnoldi basis (opt.ncv or max(2 nev + 2, 20) vectors), the GMRES basis
 * and the reduction scratch. */
int nfs_reserve(nfs_ctx* ctx, int nev);

/* Gradient of sum_j weights[j] * omega_j with respect to every per-component
 * permittivity and chirality value, from eigenvectors Y (device complex128
 * [m][4n], e.g. from nfs_eigs).  By first-order perturbation of the Hermitian
 * pencil, d omega = y^* (dA_r) y / (y^* B_r y); dA_r follows from eq.
 * factor_mtx.  Requires mu = 1.
 *   weights: HOST, m doubles.
 *   d_eps:   DEVICE, [3][n3][n2][n1] doubles (written, not accumulated).
 *   d_gamma: DEVICE, chiral [3][n3][n2][n1]; pseudochiral [n3][n2][n1].
 * Either output may be NULL.  The sum over a degenerate cluster is only
 * defined if the cluster is complete within Y. */
int nfs_eig_grad(nfs_ctx* ctx, int m, const double* weights, const void* Y,
                 double* d_eps, double* d_gamma);

/* Fields of eigenvectors (Algorithm 1, final step):
 *   x_j = [E; H] = B^{-1} diag(P_r, Q_r) y_j,  B = i [[zeta_d, mu_d], [-eps_d, -xi_d]]
 * (eq. mtx_B).  For an eigenpair (omega, y) of the HHPD-NFGEP, (omega, x) is
 * an eigenpair of the GEP diag(C, C^*) x = omega B x (eq. discrete_GEP_EH),
 * Bloch twist included: E and H are the fields on the Yee grid themselves.
 *   Y: DEVICE complex128 [m][4n] (e.g. from nfs_eigs), any scaling.
 *   X: DEVICE complex128 [m][6][n3][n2][n1], components E_x, E_y, E_z, H_x,
 *      H_y, H_z.
 * Both 16-byte aligned.  Computed in FP64 on every context; stream-ordered on
 * opt.stream (no host synchronisation).  Single-problem contexts only
 * (NFS_EUNSUPPORTED for the classes of a batch). */
int nfs_eig_fields(nfs_ctx* ctx, int m, const void* Y, void* X);

/* Relative residuals of eigenpairs of the GEP (eq. discrete_GEP_EH):
 *   res[j] = ||diag(C, C^*) x_j - omega_j B x_j||_2 / (|omega_j| ||B x_j||_2),
 * with the Yee curl C applied as its finite-difference stencil (eqs. mtx_C,
 * mtx_C123, mtx_K_n1), independent of the FFT factorisation.
 *   omega: HOST, m nonzero doubles.  X: DEVICE complex128 [m][6n] as written
 *   by nfs_eig_fields.  res: HOST, m doubles.
 * Synchronises opt.stream.  Single-problem contexts only. */
int nfs_gep_residual(nfs_ctx* ctx, int m, const double* omega, const void* X, double* res);

/* ---- media outside the Assumption: the NFSEP (Algorithm 1, 2nd branch) --
 *
 * For a nonsingular B that violates the Assumption (loss, non-reciprocal or
 * strong magnetoelectric coupling) the HHPD-NFGEP does not apply; the GEP's
 * nonzero eigenvalues are those of the null space free standard problem
 * (thm:nfep, eq. NFSEP_org)
 *   M y = omega y,  M = diag(S Q_r^*, S P_r^*) B^{-1} diag(P_r S, Q_r S),
 *   S = Sigma_r^{1/2},
 * which is not Hermitian; its eigenvalues are complex in general.  These
 * calls work in complex128 throughout. */

/* Bi-isotropic medium: per component and voxel, complex arrays [3][n3][n2][n1]
 * stored as interleaved (re, im) doubles; xi = chi + i gamma and
 * zeta = chi - i gamma (chi = 0 is the chiral medium of nfs_material). */
typedef struct {
  const double* eps;    /* permittivity                                        */
  const double* mu;     /* permeability, or NULL meaning 1                     */
  const double* gamma;  /* chirality parameter                                 */
  const double* chi;    /* Tellegen parameter, or NULL meaning 0               */
} nfs_biiso_material;

/* Set up a context for a bi-isotropic medium (grid, lattice, k and opt as
 * for nfs_setup; the material is copied).  Stores B^{-1} per voxel as one
 * 2 x 2 complex block per component; NFS_EINVAL if B is singular anywhere.
 * Only the nfs_nfsep_* calls (and nfs_destroy) apply to such a context; the
 * A_r calls return NFS_EUNSUPPORTED. */
int nfs_setup_biiso(nfs_ctx** out, const int grid[3], const double* lattice, const double k[3],
                    const nfs_biiso_material* mat, const nfs_options* opt);

/* My = M y (eq. NFSEP_org).  y, My: DEVICE complex128, 4n each, in the
 * layout of nfs_matvec's vectors, 16-byte aligned, distinct.  Stream-ordered
 * on opt.stream. */
int nfs_nfsep_matvec(nfs_ctx* ctx, const void* y, void* My);

typedef struct {
  int arnoldi_steps;          /* shift-inverted operator applications         */
  int restarts;               /* Krylov-Schur restarts                         */
  long long gmres_iterations; /* products inside the GMRES solves              */
  int nconv;                  /* wanted Ritz pairs that met eig_tol            */
  double max_ritz_residual;   /* max over them of the relative Ritz residual   */
  int status;                 /* NFS_OK or NFS_ENOCONV                          */
  long long kernel_launches;
} nfs_nfsep_info;

/* The nev eigenvalues of M nearest the complex shift sigma = {re, im}:
 * Krylov-Schur Arnoldi on (M - sigma I)^{-1} (shift-and-invert Arnoldi,
 * Section 4), each inverse applied by restarted GMRES(100) to a relative
 * residual of opt.cg_tol (at most opt.cg_maxit products); basis opt.ncv or
 * max(2 nev + 2, 20); Ritz pairs accepted at opt.eig_tol.
 *   omega: HOST, 2 nev doubles (re, im), nearest sigma first.
 *   Y:     DEVICE complex128 [nev][4n] unit eigenvectors y of M, or NULL.
 * Synchronises opt.stream; allocates the Arnoldi and GMRES bases on first
 * use unless nfs_reserve(ctx, nev) did.  Returns NFS_ENOCONV with the results
 * written if the restart cap is hit, and NFS_ENOCONV with nothing written
 * (info->status too) if an inner GMRES solve reaches opt.cg_maxit products. */
int nfs_nfsep_eigs(nfs_ctx* ctx, int nev, const double sigma[2], double* omega, void* Y, nfs_nfsep_info* info);

/* Fields of NFSEP eigenvectors (Algorithm 1, second branch): y <- S y, then
 * x = [E; H] = B^{-1} diag(P_r, Q_r) y, Bloch twist included.
 *   Y: DEVICE complex128 [m][4n];  X: DEVICE complex128 [m][6][n3][n2][n1]. */
int nfs_nfsep_fields(nfs_ctx* ctx, int m, const void* Y, void* X);

/* ---- allocation-free product ------------------------------------------ */

/* Largest voxel count n1*n2*n3 that nfs_matvec_noalloc accepts (32^3). */
#define NFS_NOALLOC_MAX_VOXELS 32768

/* Au = A_r u, like nfs_matvec, without allocating any device memory.  The
 * paper has no counterpart: this entry point is for callers that cannot
 * allocate, such as a host framework that has already reserved the GPU
 * through its own caching allocator (a raw cudaMalloc there can fail or
 * fragment its pool) or a service with a fixed device-memory budget that must
 * not allocate after start-up.  It needs no context: every input is an
 * argument.
 *   grid, k           as for nfs_setup, unit cube lattice (a = 1), mu = 1;
 *                     n1*n2*n3 <= NFS_NOALLOC_MAX_VOXELS, else NFS_EUNSUPPORTED
 *   kind, axis_a/b    NFS_MEDIUM_* and the pseudochiral pair (ignored for chiral)
 *   eps, gamma        DEVICE arrays, layout of nfs_material
 *   alpha, beta       basis parameters (eq. mtx_Lambda_p_q), e.g. 2 and 3
 *   u, Au             DEVICE complex128, 4n each, not overlapping
 *   stream            cudaStream_t (NULL = default stream)
 * Workspace: one fixed device array of 4,731,136 bytes (4.5 MiB) inside the library,
 * created when the library's device code is loaded and held by every GPU
 * that loads it until the process exits.  The first call on a device looks up
 * that array's device address and sets the kernels' shared-memory limits;
 * make that first call before any stream capture.  All calls share the one
 * array, so calls that overlap on the GPU (two streams, two host threads)
 * race and must be serialised by the caller.  The call is synchronous with
 * respect to `stream`: it returns after Au is written.  Returns NFS_ENOTHPD if
 * Phi = eps - gamma^2 <= 0 at some voxel and NFS_EINVAL if an eps or gamma is
 * not finite (Au is then meaningless; the next call starts from a cleared
 * status), and the Lemma's NFS_EKPOINT / NFS_EBASIS like nfs_setup. */
int nfs_matvec_noalloc(const int grid[3], const double k[3], int kind, int axis_a, int axis_b,
                       const double* eps, const double* gamma, double alpha, double beta,
                       const void* u, void* Au, void* stream);

/* ---- batches of independent problems ------------------------------------ */

/* A band structure (Section 5.3 sweeps k along G-X-M-R-G) is a set of
 * independent eigenproblems.  A batch solves many of them at once: problems
 * that share a grid (and medium kind, pseudochiral axis pair and mu-ness) form
 * one class whose P problems run through every kernel in single launches, in
 * lock-step, with the CG iterations replayed from a captured CUDA graph; the
 * classes run concurrently, one host thread and stream each. */
typedef struct nfs_batch nfs_batch;

typedef struct {
  int grid[3];           /* as for nfs_setup; unit cube lattice (a = 1)            */
  double k[3];           /* Bloch vector / 2 pi                                      */
  nfs_material mat;      /* host pointers, copied by nfs_setup_batch                 */
} nfs_problem;

/* Validate and set up nprob problems (the checks of nfs_setup apply to each).
 * opt as for nfs_setup (shared by all problems; its stream orders the batch
 * after earlier work).  On error *out is NULL. */
int nfs_setup_batch(nfs_batch** out, int nprob, const nfs_problem* probs, const nfs_options* opt);

/* The nev smallest positive eigenvalues of every problem, as nfs_eigs.
 * omega: HOST [nprob][nev]; info: HOST [nprob] or NULL.  Returns the worst
 * status (NFS_ENOCONV if any problem hit the restart cap). */
int nfs_eigs_batch(nfs_batch* b, int nev, double* omega, nfs_eigs_info* info);

/* Band structure: the nev smallest positive eigenvalues at each of nk Bloch
 * vectors for one grid and one medium (the k sweeps of Section 5.3).  The
 * k-points are solved in chunks, each chunk one batch (nfs_setup_batch,
 * nfs_eigs_batch: one grid class, P problems in lock-step), as many per chunk
 * as 80% of the free device memory holds with the full Lanczos basis of every
 * problem (so no problem restarts), at most max_chunk if max_chunk > 0.
 * Every k-point starts from its own random vector: starting Lanczos from the
 * previous k-point's eigenvectors saves too few steps to be worth the risk of
 * missing a band that enters from above.
 *   grid, mat, opt: as for nfs_setup_batch (unit cube lattice).
 *   k:      HOST [nk][3], Bloch vectors / 2 pi.
 *   omega:  HOST [nk][nev], ascending per k-point.
 *   info:   HOST [nk] or NULL.  chunks: HOST, the number of batches run, or NULL.
 * Returns the worst status as nfs_eigs_batch; on an error in a chunk the rows
 * of the earlier chunks are already written. */
int nfs_band_structure(const int grid[3], const nfs_material* mat, int nk, const double* k,
                       const nfs_options* opt, int nev, int max_chunk, double* omega,
                       nfs_eigs_info* info, int* chunks);

/* Number of grid classes the batch was split into. */
int nfs_batch_num_classes(const nfs_batch* b);

void nfs_destroy_batch(nfs_batch* b);

/* Basic facts about a context: n, and device bytes held. */
long long nfs_num_voxels(const nfs_ctx* ctx);
long long nfs_device_bytes(const nfs_ctx* ctx);

/* Replace the stream used by later calls (cudaStream_t). */
int nfs_set_stream(nfs_ctx* ctx, void* stream);

void nfs_destroy(nfs_ctx* ctx);
const char* nfs_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* NFS_H */
