// Host-side entry points of the three-pass A_r product (matvec_kernels.cuh),
// instantiated for complex64 (matvec_f32.cu) and complex128 (matvec_f64.cu).
#pragma once
#include <cuda_runtime.h>

#include "nfs_complex.cuh"

namespace nfs {

template <typename R>
struct MatView;

// Strides between the problems of a batched launch (P problems of one grid,
// stored back to back): elements for vectors / fields / tables, reals for the
// material, ints for the skip flags, doubles for the per-problem CG state.
struct BatchStrides {
  long long su = 0;      // u, Au, cg_r
  long long sfld = 0;    // fld
  long long smat = 0;    // inv_phi, gam, inv_mu
  long long sstate = 0;  // cg_beta, dot_part
  long long sbasis = 0;  // basis
  int slam = 0;          // lam
  int sskip = 0;         // skip
};

struct CGState;

// CG step fused into pass 3 (cluster form): instead of writing A_r p, pass 3
// forms x += alpha p and r -= alpha A_r p per voxel with alpha = rr / p^*A p
// (from pass 2's partials), and its last CTA the new r^* r, beta and the
// convergence state (the separate x/r update kernel is then not launched).
template <typename R>
struct CgFuse {
  cplx<R>* x = nullptr;
  cplx<R>* r = nullptr;
  const cplx<R>* p = nullptr;
  CGState* st = nullptr;  // per problem: st + prob
};

template <typename R>
struct MatvecArgs {
  const cplx<R>* u;       // 4n, spectral
  cplx<R>* Au;            // 4n, spectral
  cplx<R>* fld;           // 6n workspace
  const cplx<R>* lam;     // Lambda_1 | Lambda_2 | Lambda_3 (n1 + n2 + n3)
  const cplx<R>* tw1;     // exp(-2 pi i m / n1), m < n1
  const cplx<R>* tw2;
  const cplx<R>* tw3;
  const R* inv_phi;
  const R* gam;
  const R* inv_mu;        // nullptr for mu = 1
  int kind, ax_a, ax_b;
  int n1, n2, n3;
  R alpha, beta;
  const int* skip;        // device flag: when nonzero every pass returns at once
  // optional table of the per-voxel basis, [c_x, c_y, c_z, x_x, x_y, x_z][n]
  // (spectral order); nullptr: evaluated from the Lambda tables in the kernels
  const cplx<R>* basis;
  cudaStream_t stream;
  // CG fusion (both optional, nullptr when unused):
  const cplx<R>* cg_r;    // pass 1 first forms p = cg_r + (*cg_beta) u ...
  const double* cg_beta;
  cplx<R>* p_out;         // ... and stores it here (nullptr: in place, into u; the
                          // paired complex64 kernels need a separate buffer)
  double* dot_part;       // one partial of Re(u^* A u) per CTA of pass 2 (pass 3b in the five-pass form)
  CgFuse<R> cg;           // optional: the CG step fused into pass 3 (see cg_fusable)
  // batching: P problems of this grid in one launch (P = 1 for one problem)
  int P;
  BatchStrides bs;
};

// Largest dynamic shared memory a CTA may request on sm_103a.
constexpr size_t kMaxDynSmem = 232448;

// Whether the kernels exist for this grid in this precision (n1 = n2 and each
// size in {8, 12, 16, 24, 32, 48, 64, 96, 128}, plane fits in shared memory).
template <typename R> bool matvec_supported(int n1, int n2, int n3);
// Opt the chosen kernels in to their dynamic shared memory (once per device).
template <typename R> cudaError_t matvec_prepare(int n1, int n2, int n3);
template <typename R> cudaError_t matvec_launch(const MatvecArgs<R>& a);
// Selected passes only (bit 0: pass 1, bit 1: pass 2, bit 2: pass 3).
template <typename R> cudaError_t matvec_launch_mask(const MatvecArgs<R>& a, int mask);
// Split launches used by the eigenvector-gradient path: pass 1 only.
template <typename R> cudaError_t pass1_launch(const MatvecArgs<R>& a);
// Kernels one plane pass launches for grids n1 x n1 (1 cluster form, 2 five-pass form).
template <typename R> int plane_pass_kernels(int n1);
// Kernels one whole product launches for grids n1 x n1.
template <typename R> int product_kernels(int n1);
// Whether the CG direction update of pass 1 needs p_out distinct from u
// (the paired complex64 plane kernels read every voxel of u in three CTAs).
template <typename R> bool cg_needs_p_out(int n1);
// Whether pass 3 can take the CG step (MatvecArgs::cg) for grids n1 x n1.
template <typename R> bool cg_fusable(int n1);
// Number of p^* A p partials a CG product emits per problem (dot_part entries).
template <typename R> int matvec_dot_partials(int n1, int n2, int n3);

// The basis table for MatvecArgs<double>::basis: P problems (Lambda tables
// at lam + p * slam, tables at basis + p * sbasis).
cudaError_t basis_table_launch(const double2* lam, int n1, int n2, int n3, double alpha, double beta, double2* basis,
                               int P, int slam, long long sbasis, cudaStream_t stream);

// Double-single element conversions (matvec_df.cu); `count` reals, in and out
// may alias for df_to_double.
struct df;
cudaError_t double_to_df(const double* in, df* out, long long count, cudaStream_t s);
cudaError_t df_to_double(const df* in, double* out, long long count, cudaStream_t s);

// Gradient accumulation (complex128 only): inverse z-DFT of the six pass-1
// fields and, per voxel, d_eps += scale * dA/deps, d_gamma += scale * dA/dgamma.
struct GradArgs {
  const double2* fld;
  const double2* tw3;
  const double* inv_phi;
  const double* gam;
  int kind, ax_a, ax_b;
  int n1, n2, n3;
  double scale;
  double* d_eps;
  double* d_gamma;
  cudaStream_t stream;
};
cudaError_t grad_prepare(int n1, int n2, int n3);
cudaError_t grad_launch(const GradArgs& a);

// Fields [E; H] = B^{-1} diag(P_r, Q_r) y of one eigenvector from the pass-1
// fields of y (matvec_f64.cu).
struct FieldsArgs {
  const double2* fld;     // pass-1 output, 6n
  const double2* tw3;
  const double2* bloch;   // D_1 | D_2 | D_3 diagonals, n1 + n2 + n3
  const double* inv_phi;
  const double* gam;
  const double* inv_mu;   // nullptr for mu = 1
  int kind, ax_a, ax_b;
  int n1, n2, n3;
  double2* X;             // 6n out: E_x, E_y, E_z, H_x, H_y, H_z
  cudaStream_t stream;
};
cudaError_t fields_prepare(int n1, int n2, int n3);
cudaError_t fields_launch(const FieldsArgs& a);

// Partial sums of the GEP residual of (omega, x) (matvec_f64.cu).
struct GepResidualArgs {
  const double2* X;       // 6n: E_x, E_y, E_z, H_x, H_y, H_z
  const double* inv_phi;
  const double* gam;
  const double* inv_mu;   // nullptr for mu = 1
  int kind, ax_a, ax_b;
  int n1, n2, n3;
  double inv_delta[3];
  double2 wrap[3];        // exp(i 2 pi k.a_l)
  double omega;
  double* part;           // 2 per block: |residual|^2, |B x|^2
};
cudaError_t gep_residual_launch(const GepResidualArgs& a, int blocks, cudaStream_t stream);

}  // namespace nfs
