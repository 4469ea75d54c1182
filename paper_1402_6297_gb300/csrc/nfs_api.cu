// libnfs C ABI: context setup, A_r and B_r products, CG (FP64 and mixed
// precision with FP64 refinement), thick-restart invert Lanczos on the
// HHPD-NFGEP, and the eigenvalue gradient.  See include/nfs.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/nfs.h"
#include "blas_kernels.cuh"
#include "matvec.h"

using nfs::CGState;
using nfs::kRedBlocks;
using nfs::kRedThreads;

struct nfs_ctx {
  int n1 = 0, n2 = 0, n3 = 0;
  long long n = 0, N = 0;  // voxels, 4n
  double kdota[3] = {0, 0, 0};
  double delta[3] = {0, 0, 0};
  nfs_options opt{};
  cudaStream_t stream = nullptr;
  int kind = 0, ax_a = 0, ax_b = 1;
  bool has_mu = false;
  // tables
  double2* lam64 = nullptr;
  float2* lam32 = nullptr;
  double2* tw64[3] = {nullptr, nullptr, nullptr};
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  // material: inv_phi [3n] | gam [3n or n] | inv_mu [3n] (optional)
  double* mat64 = nullptr;
  float* mat32 = nullptr;
  long long gam_len = 0;
  // workspaces
  void* fld = nullptr;  // 6n complex128 (complex64 uses the first half)
  double2 *x64 = nullptr, *r64 = nullptr, *p64 = nullptr, *Ap64 = nullptr, *t64 = nullptr, *t64b = nullptr;
  float2 *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *Ap32 = nullptr;
  CGState* st = nullptr;
  CGState* st_host = nullptr;  // pinned mirror (done/it/status/rr)
  double* dscratch = nullptr;  // reductions
  size_t dscratch_len = 0;
  double* hscratch = nullptr;  // pinned
  size_t hscratch_len = 0;
  // Lanczos basis
  double2* V = nullptr;
  double2* MV = nullptr;
  int vcap = 0;
  double* dY = nullptr;  // rotation coefficients
  int dY_len = 0;
  long long bytes = 0;
  long long mv32 = 0, mv64 = 0;
};

namespace {

thread_local char g_errbuf[256];

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_errbuf, sizeof(g_errbuf), "%s: %s", what, cudaGetErrorString(e));
  return NFS_ECUDA;
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);            \
  } while (0)

template <typename T>
int dalloc(nfs_ctx* c, T** p, size_t count) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return NFS_ENOMEM;
  }
  c->bytes += (long long)bytes;
  return NFS_OK;
}

#define TRY(call)                 \
  do {                            \
    int r_ = (call);              \
    if (r_ != NFS_OK) return r_;  \
  } while (0)

bool size_ok(int s) {
  switch (s) {
    case 8: case 12: case 16: case 24: case 32: case 48: case 64: case 96: case 128: return true;
    default: return false;
  }
}

int grid_blocks(long long N, int threads) {
  long long b = (N + threads - 1) / threads;
  return (int)std::min<long long>(b, 152LL * 16);
}

// --- matvec -------------------------------------------------------------

template <typename R>
nfs::MatvecArgs<R> margs(nfs_ctx* c, const nfs::cplx<R>* u, nfs::cplx<R>* Au, const int* skip);

template <>
nfs::MatvecArgs<double> margs<double>(nfs_ctx* c, const double2* u, double2* Au, const int* skip) {
  nfs::MatvecArgs<double> a{};
  a.u = u; a.Au = Au; a.fld = (double2*)c->fld; a.lam = c->lam64;
  a.tw1 = c->tw64[0]; a.tw2 = c->tw64[1]; a.tw3 = c->tw64[2];
  a.inv_phi = c->mat64; a.gam = c->mat64 + 3 * c->n; a.inv_mu = c->has_mu ? c->mat64 + 3 * c->n + c->gam_len : nullptr;
  a.kind = c->kind; a.ax_a = c->ax_a; a.ax_b = c->ax_b;
  a.n1 = c->n1; a.n2 = c->n2; a.n3 = c->n3; a.alpha = c->opt.alpha; a.beta = c->opt.beta;
  a.skip = skip; a.stream = c->stream;
  return a;
}

template <>
nfs::MatvecArgs<float> margs<float>(nfs_ctx* c, const float2* u, float2* Au, const int* skip) {
  nfs::MatvecArgs<float> a{};
  a.u = u; a.Au = Au; a.fld = (float2*)c->fld; a.lam = c->lam32;
  a.tw1 = c->tw32[0]; a.tw2 = c->tw32[1]; a.tw3 = c->tw32[2];
  a.inv_phi = c->mat32; a.gam = c->mat32 + 3 * c->n; a.inv_mu = c->has_mu ? c->mat32 + 3 * c->n + c->gam_len : nullptr;
  a.kind = c->kind; a.ax_a = c->ax_a; a.ax_b = c->ax_b;
  a.n1 = c->n1; a.n2 = c->n2; a.n3 = c->n3; a.alpha = (float)c->opt.alpha; a.beta = (float)c->opt.beta;
  a.skip = skip; a.stream = c->stream;
  return a;
}

template <typename R>
int matvec(nfs_ctx* c, const nfs::cplx<R>* u, nfs::cplx<R>* Au, const int* skip = nullptr) {
  cudaError_t e = nfs::matvec_launch<R>(margs<R>(c, u, Au, skip));
  if (e != cudaSuccess) return cuda_fail(e, "matvec launch");
  if (sizeof(R) == 4) c->mv32++; else c->mv64++;
  return NFS_OK;
}

// --- reductions -------------------------------------------------------------

template <typename C>
int dot_re(nfs_ctx* c, const C* x, const C* y, double* out) {
  nfs::k_dot_re<C><<<kRedBlocks, kRedThreads, 0, c->stream>>>(x, y, c->N, c->dscratch, nullptr);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->hscratch, c->dscratch, kRedBlocks * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double s = 0.0;
  for (int i = 0; i < kRedBlocks; ++i) s += c->hscratch[i];
  *out = s;
  return NFS_OK;
}

// --- CG ---------------------------------------------------------------------

constexpr int kCgChunk = 8;

// Runs CG from the state r = b - A x (already formed), p scratch.  tol2 is the
// absolute threshold on r^* r.  Returns NFS_OK / NFS_E* and the iteration count.
template <typename R>
int cg_run(nfs_ctx* c, nfs::cplx<R>* x, nfs::cplx<R>* r, nfs::cplx<R>* p, nfs::cplx<R>* Ap, double tol2, int maxit,
           int* iters, int* status) {
  using C = nfs::cplx<R>;
  const long long N = c->N;
  CK(cudaMemcpyAsync(p, r, N * sizeof(C), cudaMemcpyDeviceToDevice, c->stream));
  nfs::k_dot_re<C><<<kRedBlocks, kRedThreads, 0, c->stream>>>(r, r, N, c->st->part_a, nullptr);
  nfs::k_cg_init<<<1, kRedThreads, 0, c->stream>>>(c->st, tol2, maxit);
  CK(cudaGetLastError());
  int done = 0;
  const int* skip = &c->st->done;
  for (;;) {
    for (int i = 0; i < kCgChunk; ++i) {
      TRY(matvec<R>(c, p, Ap, skip));
      nfs::k_dot_re<C><<<kRedBlocks, kRedThreads, 0, c->stream>>>(p, Ap, N, c->st->part_a, skip);
      nfs::k_cg_alpha<<<1, kRedThreads, 0, c->stream>>>(c->st);
      nfs::k_cg_update_xr<C><<<kRedBlocks, kRedThreads, 0, c->stream>>>(x, r, p, Ap, N, c->st);
      nfs::k_cg_beta<<<1, kRedThreads, 0, c->stream>>>(c->st);
      nfs::k_cg_update_p<C><<<kRedBlocks, kRedThreads, 0, c->stream>>>(p, r, N, c->st);
      CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(c->st_host, c->st, offsetof(CGState, part_a), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    done = c->st_host->done;
    if (done) break;
  }
  *iters = c->st_host->it;
  *status = c->st_host->status;
  return NFS_OK;
}

int launch_sub64(nfs_ctx* c, const double2* a, const double2* b, double2* y) {
  nfs::k_sub<double2><<<grid_blocks(c->N, 256), 256, 0, c->stream>>>(a, b, y, c->N);
  CK(cudaGetLastError());
  return NFS_OK;
}

// FP64 CG on A_r x = b (complex128 throughout).
int solve_fp64(nfs_ctx* c, const double2* b, double2* x, bool x_zero, nfs_solve_info* info) {
  double bb;
  TRY(dot_re(c, b, b, &bb));
  if (bb == 0.0) {
    CK(cudaMemsetAsync(x, 0, c->N * sizeof(double2), c->stream));
    if (info) *info = nfs_solve_info{0, 0, 0.0, NFS_OK};
    return NFS_OK;
  }
  if (x_zero) {
    CK(cudaMemsetAsync(x, 0, c->N * sizeof(double2), c->stream));
    CK(cudaMemcpyAsync(c->r64, b, c->N * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    TRY(matvec<double>(c, x, c->Ap64));
    TRY(launch_sub64(c, b, c->Ap64, c->r64));
  }
  int it = 0, st = 0;
  const double tol = c->opt.cg_tol;
  TRY(cg_run<double>(c, x, c->r64, c->p64, c->Ap64, tol * tol * bb, c->opt.cg_maxit, &it, &st));
  if (info) {
    info->iterations = it;
    info->refinements = 0;
    info->rel_residual = std::sqrt(std::max(c->st_host->rr, 0.0) / bb);
    info->status = st;
  }
  return st;
}

// Mixed precision: complex64 CG inner solves inside FP64 iterative refinement
// r = b - A_r x evaluated with the complex128 product.
int solve_mixed(nfs_ctx* c, const double2* b, double2* x, bool x_zero, nfs_solve_info* info) {
  double bb;
  TRY(dot_re(c, b, b, &bb));
  if (bb == 0.0) {
    CK(cudaMemsetAsync(x, 0, c->N * sizeof(double2), c->stream));
    if (info) *info = nfs_solve_info{0, 0, 0.0, NFS_OK};
    return NFS_OK;
  }
  if (x_zero) {
    CK(cudaMemsetAsync(x, 0, c->N * sizeof(double2), c->stream));
    CK(cudaMemcpyAsync(c->r64, b, c->N * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    TRY(matvec<double>(c, x, c->Ap64));
    TRY(launch_sub64(c, b, c->Ap64, c->r64));
  }
  const double tol2 = c->opt.cg_tol * c->opt.cg_tol * bb;
  int total_it = 0, refines = 0, status = NFS_OK;
  double rr = 0.0;
  const int nb = grid_blocks(c->N, 256);
  for (;;) {
    TRY(dot_re(c, c->r64, c->r64, &rr));
    if (!(rr == rr)) { status = NFS_EBREAKDOWN; break; }
    if (rr <= tol2) break;
    if (refines >= c->opt.max_refine) { status = NFS_ENOCONV; break; }
    const double rn = std::sqrt(rr);
    nfs::k_demote<<<nb, 256, 0, c->stream>>>(c->r64, 1.0 / rn, c->r32, c->N);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(c->x32, 0, c->N * sizeof(float2), c->stream));
    int it = 0, st = 0;
    const double itol = c->opt.inner_tol;
    TRY(cg_run<float>(c, c->x32, c->r32, c->p32, c->Ap32, itol * itol, c->opt.cg_maxit, &it, &st));
    total_it += it;
    nfs::k_axpy_promote<<<nb, 256, 0, c->stream>>>(x, rn, c->x32, c->N);
    CK(cudaGetLastError());
    TRY(matvec<double>(c, x, c->Ap64));
    TRY(launch_sub64(c, b, c->Ap64, c->r64));
    ++refines;
    if (st == NFS_EBREAKDOWN) { status = st; break; }
  }
  if (info) {
    info->iterations = total_it;
    info->refinements = refines;
    info->rel_residual = std::sqrt(std::max(rr, 0.0) / bb);
    info->status = status;
  }
  return status;
}

int solve(nfs_ctx* c, const double2* b, double2* x, bool x_zero, nfs_solve_info* info) {
  if (c->opt.precision == NFS_PREC_MIXED) return solve_mixed(c, b, x, x_zero, info);
  return solve_fp64(c, b, x, x_zero, info);
}

// --- host symmetric eigensolver (cyclic Jacobi) ------------------------------

// A (m x m, row-major, symmetric) -> eigenvalues w (ascending) and
// eigenvectors as the columns of Z (row-major m x m).
void jacobi_eig(int m, std::vector<double> A, std::vector<double>& w, std::vector<double>& Z) {
  Z.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Z[(size_t)i * m + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * m + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < m; ++i) {
      diag += a(i, i) * a(i, i);
      for (int j = i + 1; j < m; ++j) off += a(i, j) * a(i, j);
    }
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = cs * akp - sn * akq;
          a(k, q) = sn * akp + cs * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = cs * apk - sn * aqk;
          a(q, k) = sn * apk + cs * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double zkp = Z[(size_t)k * m + p], zkq = Z[(size_t)k * m + q];
          Z[(size_t)k * m + p] = cs * zkp - sn * zkq;
          Z[(size_t)k * m + q] = sn * zkp + cs * zkq;
        }
      }
    }
  }
  std::vector<int> idx(m);
  for (int i = 0; i < m; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return a(i, i) < a(j, j); });
  w.resize(m);
  std::vector<double> Zs((size_t)m * m);
  for (int c2 = 0; c2 < m; ++c2) {
    w[c2] = a(idx[c2], idx[c2]);
    for (int k = 0; k < m; ++k) Zs[(size_t)k * m + c2] = Z[(size_t)k * m + idx[c2]];
  }
  Z.swap(Zs);
}

int ensure_scratch(nfs_ctx* c, size_t dlen) {
  if (c->dscratch_len < dlen) {
    if (c->dscratch) cudaFree(c->dscratch);
    c->dscratch = nullptr;
    TRY(dalloc(c, &c->dscratch, dlen));
    c->dscratch_len = dlen;
  }
  if (c->hscratch_len < dlen) {
    if (c->hscratch) cudaFreeHost(c->hscratch);
    c->hscratch = nullptr;
    CK(cudaMallocHost((void**)&c->hscratch, dlen * sizeof(double)));
    c->hscratch_len = dlen;
  }
  return NFS_OK;
}

// Lanczos scratch layout in dscratch (mcap = basis capacity):
//   [0, P)            per-block partial dots, P = kRedBlocks * 2 * mcap
//   [P, P + 2 mcap)   finished dots
//   [P + 2 mcap, ...) coefficients for the update
size_t lanczos_scratch_len(int mcap) { return (size_t)kRedBlocks * 2 * mcap + 4 * (size_t)mcap + 64; }

// c = V[0:m]^* w (complex, m entries) on the host
int multi_dot(nfs_ctx* c, const double2* V, int m, const double2* w, std::vector<double>& out) {
  double* part = c->dscratch;
  double* fin = c->dscratch + (size_t)kRedBlocks * 2 * c->vcap;
  nfs::k_multi_dot<kRedThreads><<<kRedBlocks, kRedThreads, 0, c->stream>>>(V, m, w, c->N, part);
  nfs::k_multi_dot_finish<<<m, kRedThreads, 0, c->stream>>>(part, m, kRedBlocks, fin);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->hscratch, fin, (size_t)m * 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  out.assign(c->hscratch, c->hscratch + 2 * m);
  return NFS_OK;
}

int multi_axpy(nfs_ctx* c, double2* w, double2* Mw, const double2* V, const double2* MV, int m,
               const std::vector<double>& coef) {
  double* dcoef = c->dscratch + (size_t)kRedBlocks * 2 * c->vcap + 2 * (size_t)c->vcap;
  std::memcpy(c->hscratch, coef.data(), coef.size() * sizeof(double));
  CK(cudaMemcpyAsync(dcoef, c->hscratch, coef.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  nfs::k_multi_axpy<<<grid_blocks(c->N, 256), 256, 0, c->stream>>>(w, Mw, V, MV, dcoef, m, c->N);
  CK(cudaGetLastError());
  // the host scratch is reused by the next call: make sure the copy consumed it
  CK(cudaStreamSynchronize(c->stream));
  return NFS_OK;
}

int ensure_basis(nfs_ctx* c, int m) {
  if (c->vcap >= m + 1) return NFS_OK;
  if (c->V) { cudaFree(c->V); c->bytes -= (long long)c->vcap * c->N * 16; c->V = nullptr; }
  if (c->MV) { cudaFree(c->MV); c->bytes -= (long long)c->vcap * c->N * 16; c->MV = nullptr; }
  c->vcap = 0;
  TRY(dalloc(c, &c->V, (size_t)(m + 1) * c->N));
  TRY(dalloc(c, &c->MV, (size_t)(m + 1) * c->N));
  c->vcap = m + 1;
  return NFS_OK;
}

// V[0:k] = V[0:m] Y (Y real m x k column-major)
int rotate(nfs_ctx* c, double2* V, int m, const std::vector<double>& Ycm, int k) {
  if (c->dY_len < m * k) {
    if (c->dY) cudaFree(c->dY);
    c->dY = nullptr;
    TRY(dalloc(c, &c->dY, (size_t)m * k));
    c->dY_len = m * k;
  }
  CK(cudaMemcpyAsync(c->dY, Ycm.data(), (size_t)m * k * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  constexpr int TE = 32;
  const size_t smem = (size_t)m * TE * sizeof(double2);
  CK(cudaFuncSetAttribute(nfs::k_rotate_basis<TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  nfs::k_rotate_basis<TE><<<grid_blocks((c->N + TE - 1) / TE, 1), 256, smem, c->stream>>>(V, m, c->dY, k, c->N);
  CK(cudaGetLastError());
  return NFS_OK;
}

int apply_Br(nfs_ctx* c, const double2* v, double2* out) {
  nfs::k_apply_Br<<<grid_blocks(c->n, 256), 256, 0, c->stream>>>(v, out, c->lam64, c->n1, c->n2, c->n3);
  CK(cudaGetLastError());
  return NFS_OK;
}

void free_ctx(nfs_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->lam64, c->lam32, c->tw64[0], c->tw64[1], c->tw64[2], c->tw32[0], c->tw32[1], c->tw32[2],
                  c->mat64, c->mat32, c->fld, c->x64, c->r64, c->p64, c->Ap64, c->t64, c->t64b, c->x32, c->r32,
                  c->p32, c->Ap32, c->st, c->dscratch, c->V, c->MV, c->dY};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->hscratch) cudaFreeHost(c->hscratch);
  delete c;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" void nfs_default_options(nfs_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = NFS_PREC_FP64;
  o->alpha = 2.0;
  o->beta = 3.0;
  o->cg_tol = 1e-12;
  o->cg_maxit = 2000;
  o->inner_tol = 1e-5;
  o->max_refine = 8;
  o->eig_tol = 1e-10;
  o->ncv = 0;
  o->max_restarts = 200;
  o->seed = 1;
  o->stream = nullptr;
}

extern "C" const char* nfs_strerror(int code) {
  switch (code) {
    case NFS_OK: return "ok";
    case NFS_EINVAL: return "invalid argument";
    case NFS_EUNSUPPORTED: return "unsupported grid or lattice";
    case NFS_EKPOINT: return "k.a_l all integers: Lambda_q is singular";
    case NFS_EBASIS: return "alpha, beta make Lambda_p rank deficient";
    case NFS_ENOTHPD: return "mu or Phi = eps - xi mu^-1 zeta not positive definite";
    case NFS_ENOCONV: return "iteration limit reached";
    case NFS_EBREAKDOWN: return "breakdown (non-positive curvature or NaN)";
    case NFS_ETIMEOUT: return "device wait timed out";
    case NFS_ECUDA: return g_errbuf[0] ? g_errbuf : "CUDA error";
    case NFS_ENOMEM: return "device allocation failed";
    default: return "unknown error";
  }
}

extern "C" int nfs_setup(nfs_ctx** out, const int grid[3], const double* lattice, const double k[3],
                         const nfs_material* mat, const nfs_options* opt) {
  if (!out) return NFS_EINVAL;
  *out = nullptr;
  if (!grid || !k || !mat || !mat->eps || !mat->gamma) return NFS_EINVAL;
  for (int l = 0; l < 3; ++l)
    if (grid[l] <= 0) return NFS_EINVAL;
  if (mat->kind != NFS_MEDIUM_CHIRAL && mat->kind != NFS_MEDIUM_PSEUDOCHIRAL) return NFS_EINVAL;
  if (mat->kind == NFS_MEDIUM_PSEUDOCHIRAL &&
      (mat->axis_a < 0 || mat->axis_a > 2 || mat->axis_b < 0 || mat->axis_b > 2 || mat->axis_a == mat->axis_b))
    return NFS_EINVAL;
  nfs_options o;
  nfs_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != NFS_PREC_FP64 && o.precision != NFS_PREC_MIXED) return NFS_EINVAL;
  if (!(o.cg_tol > 0) || o.cg_maxit <= 0 || !(o.eig_tol > 0) || o.max_restarts < 0) return NFS_EINVAL;
  if (o.precision == NFS_PREC_MIXED && (!(o.inner_tol > 0) || o.inner_tol >= 1 || o.max_refine <= 0))
    return NFS_EINVAL;
  if (!(o.alpha != 0.0) || !(o.beta != 0.0)) return NFS_EBASIS;

  const int n1 = grid[0], n2 = grid[1], n3 = grid[2];
  if (!size_ok(n1) || !size_ok(n2) || !size_ok(n3) || n1 != n2) return NFS_EUNSUPPORTED;
  if (!nfs::matvec_supported<double>(n1, n2, n3) || !nfs::matvec_supported<float>(n1, n2, n3))
    return NFS_EUNSUPPORTED;
  double a_len[3] = {1.0, 1.0, 1.0};
  if (lattice) {
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s)
        if (r != s && lattice[3 * r + s] != 0.0) return NFS_EUNSUPPORTED;
    for (int l = 0; l < 3; ++l) {
      a_len[l] = std::fabs(lattice[4 * l]);
      if (!(a_len[l] > 0)) return NFS_EINVAL;
    }
  }
  const long long n = (long long)n1 * n2 * n3;
  double kd[3], delta[3];
  const int nn[3] = {n1, n2, n3};
  bool all_int = true;
  for (int l = 0; l < 3; ++l) {
    if (!std::isfinite(k[l])) return NFS_EINVAL;
    kd[l] = k[l] * a_len[l];
    delta[l] = a_len[l] / nn[l];
    if (std::fabs(kd[l] - std::round(kd[l])) > 1e-12) all_int = false;
  }
  if (all_int) return NFS_EKPOINT;

  // Lambda tables (thm:SchurDecomp_Ci): (exp(i 2 pi (i + k.a)/m) - 1) / delta,
  // real part written as -2 sin^2(theta/2) to avoid cancellation.
  std::vector<double2> lam(n1 + n2 + n3);
  {
    int off = 0;
    for (int l = 0; l < 3; ++l) {
      for (int i = 0; i < nn[l]; ++i) {
        const double th = 2.0 * M_PI * (i + kd[l]) / nn[l];
        const double sh = std::sin(0.5 * th);
        lam[off + i] = make_double2(-2.0 * sh * sh / delta[l], std::sin(th) / delta[l]);
      }
      off += nn[l];
    }
  }
  // Lemma (lem:nonsingular_full_rank): Lambda_q > 0 and Lambda_p != 0 at every voxel
  {
    const double al = o.alpha, be = o.beta;
    double minq = INFINITY, minp = INFINITY;
    for (int i3 = 0; i3 < n3; ++i3)
      for (int i2 = 0; i2 < n2; ++i2)
        for (int i1 = 0; i1 < n1; ++i1) {
          const double2 a1 = lam[i1], a2 = lam[n1 + i2], a3 = lam[n1 + n2 + i3];
          const double lq = nfs::cabs2(a1) + nfs::cabs2(a2) + nfs::cabs2(a3);
          const double2 p1 = make_double2(be * a3.x - a2.x, be * a3.y - a2.y);
          const double2 p2 = make_double2(a1.x - al * a3.x, a1.y - al * a3.y);
          const double2 p3 = make_double2(al * a2.x - be * a1.x, al * a2.y - be * a1.y);
          const double lp = nfs::cabs2(p1) + nfs::cabs2(p2) + nfs::cabs2(p3);
          minq = std::min(minq, lq);
          minp = std::min(minp, lp / ((al * al + be * be + 1.0) * lq));
        }
    if (!(minq > 0)) return NFS_EKPOINT;
    if (!(minp > 1e-13)) return NFS_EBASIS;
  }

  // material (Section 4.3): 1/Phi, gamma, 1/mu per component; Assumption check
  const bool has_mu = mat->mu != nullptr;
  const long long gam_len = (mat->kind == NFS_MEDIUM_CHIRAL) ? 3 * n : n;
  const long long mat_len = 3 * n + gam_len + (has_mu ? 3 * n : 0);
  std::vector<double> m64(mat_len);
  {
    double* inv_phi = m64.data();
    double* gam = inv_phi + 3 * n;
    double* inv_mu = gam + gam_len;
    for (long long i = 0; i < gam_len; ++i) {
      if (!std::isfinite(mat->gamma[i])) return NFS_EINVAL;
      gam[i] = mat->gamma[i];
    }
    for (long long i = 0; i < 3 * n; ++i) {
      const double mu = has_mu ? mat->mu[i] : 1.0;
      if (!(mu > 0) || !std::isfinite(mu) || !std::isfinite(mat->eps[i])) return NFS_ENOTHPD;
      if (has_mu) inv_mu[i] = 1.0 / mu;
    }
    for (int cpt = 0; cpt < 3; ++cpt) {
      for (long long v = 0; v < n; ++v) {
        const long long i = cpt * n + v;
        double phi;
        if (mat->kind == NFS_MEDIUM_CHIRAL) {
          const double mu = has_mu ? mat->mu[i] : 1.0;
          phi = mat->eps[i] - gam[i] * gam[i] / mu;
        } else {
          const int a = mat->axis_a, b = mat->axis_b;
          const double g = gam[v];
          if (cpt == a) phi = mat->eps[i] - g * g / (has_mu ? mat->mu[b * n + v] : 1.0);
          else if (cpt == b) phi = mat->eps[i] - g * g / (has_mu ? mat->mu[a * n + v] : 1.0);
          else phi = mat->eps[i];
        }
        if (!(phi > 0)) return NFS_ENOTHPD;
        inv_phi[i] = 1.0 / phi;
      }
    }
  }

  int dev = 0;
  CK(cudaGetDevice(&dev));
  nfs_ctx* c = new (std::nothrow) nfs_ctx();
  if (!c) return NFS_ENOMEM;
  c->n1 = n1; c->n2 = n2; c->n3 = n3; c->n = n; c->N = 4 * n;
  for (int l = 0; l < 3; ++l) { c->kdota[l] = kd[l]; c->delta[l] = delta[l]; }
  c->opt = o;
  c->stream = (cudaStream_t)o.stream;
  c->kind = mat->kind; c->ax_a = mat->axis_a; c->ax_b = mat->axis_b;
  if (c->kind == NFS_MEDIUM_CHIRAL) { c->ax_a = 0; c->ax_b = 1; }
  c->has_mu = has_mu;
  c->gam_len = gam_len;

  auto fail = [&](int code) { free_ctx(c); return code; };
#define TRYC(call)                         \
  do {                                     \
    int r_ = (call);                       \
    if (r_ != NFS_OK) return fail(r_);     \
  } while (0)
#define CKC(call)                                               \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return fail(cuda_fail(e_, #call));   \
  } while (0)

  const int nl = n1 + n2 + n3;
  TRYC(dalloc(c, &c->lam64, nl));
  TRYC(dalloc(c, &c->lam32, nl));
  std::vector<float2> lam32(nl);
  for (int i = 0; i < nl; ++i) lam32[i] = make_float2((float)lam[i].x, (float)lam[i].y);
  CKC(cudaMemcpy(c->lam64, lam.data(), nl * sizeof(double2), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(c->lam32, lam32.data(), nl * sizeof(float2), cudaMemcpyHostToDevice));
  for (int l = 0; l < 3; ++l) {
    const int m = nn[l];
    std::vector<double2> t(m);
    std::vector<float2> t32(m);
    for (int i = 0; i < m; ++i) {
      const double th = -2.0 * M_PI * i / m;
      t[i] = make_double2(std::cos(th), std::sin(th));
      t32[i] = make_float2((float)t[i].x, (float)t[i].y);
    }
    TRYC(dalloc(c, &c->tw64[l], m));
    TRYC(dalloc(c, &c->tw32[l], m));
    CKC(cudaMemcpy(c->tw64[l], t.data(), m * sizeof(double2), cudaMemcpyHostToDevice));
    CKC(cudaMemcpy(c->tw32[l], t32.data(), m * sizeof(float2), cudaMemcpyHostToDevice));
  }
  TRYC(dalloc(c, &c->mat64, mat_len));
  TRYC(dalloc(c, &c->mat32, mat_len));
  {
    std::vector<float> m32(mat_len);
    for (long long i = 0; i < mat_len; ++i) m32[i] = (float)m64[i];
    CKC(cudaMemcpy(c->mat64, m64.data(), mat_len * sizeof(double), cudaMemcpyHostToDevice));
    CKC(cudaMemcpy(c->mat32, m32.data(), mat_len * sizeof(float), cudaMemcpyHostToDevice));
  }
  const long long N = c->N;
  TRYC(dalloc(c, (double2**)&c->fld, 6 * n));
  TRYC(dalloc(c, &c->x64, N));
  TRYC(dalloc(c, &c->r64, N));
  TRYC(dalloc(c, &c->p64, N));
  TRYC(dalloc(c, &c->Ap64, N));
  TRYC(dalloc(c, &c->t64, N));
  TRYC(dalloc(c, &c->t64b, N));
  if (o.precision == NFS_PREC_MIXED) {
    TRYC(dalloc(c, &c->x32, N));
    TRYC(dalloc(c, &c->r32, N));
    TRYC(dalloc(c, &c->p32, N));
    TRYC(dalloc(c, &c->Ap32, N));
  }
  TRYC(dalloc(c, &c->st, 1));
  CKC(cudaMallocHost((void**)&c->st_host, sizeof(CGState)));
  std::memset(c->st_host, 0, sizeof(CGState));
  CKC(cudaMemset(c->st, 0, sizeof(CGState)));
  TRYC(ensure_scratch(c, (size_t)kRedBlocks * 2 * 64 + 4096));
  CKC(nfs::matvec_prepare<double>(n1, n2, n3));
  CKC(nfs::matvec_prepare<float>(n1, n2, n3));
  CKC(nfs::grad_prepare(n1, n2, n3));
  CKC(cudaDeviceSynchronize());
#undef TRYC
#undef CKC
  *out = c;
  return NFS_OK;
}

extern "C" void nfs_destroy(nfs_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

extern "C" long long nfs_num_voxels(const nfs_ctx* c) { return c ? c->n : 0; }
extern "C" long long nfs_device_bytes(const nfs_ctx* c) { return c ? c->bytes : 0; }

extern "C" int nfs_set_stream(nfs_ctx* c, void* stream) {
  if (!c) return NFS_EINVAL;
  c->stream = (cudaStream_t)stream;
  c->opt.stream = stream;
  return NFS_OK;
}

extern "C" int nfs_matvec(nfs_ctx* c, int dtype, const void* u, void* Au) {
  if (!c || !u || !Au || u == Au) return NFS_EINVAL;
  if (dtype == NFS_C128) return matvec<double>(c, (const double2*)u, (double2*)Au);
  if (dtype == NFS_C64) return matvec<float>(c, (const float2*)u, (float2*)Au);
  return NFS_EINVAL;
}

extern "C" int nfs_matvec_passes(nfs_ctx* c, int dtype, int mask, const void* u, void* Au) {
  if (!c || mask <= 0 || mask > 7) return NFS_EINVAL;
  if ((mask & 1) && !u) return NFS_EINVAL;
  if ((mask & 4) && !Au) return NFS_EINVAL;
  cudaError_t e;
  if (dtype == NFS_C128)
    e = nfs::matvec_launch_mask<double>(margs<double>(c, (const double2*)u, (double2*)Au, nullptr), mask);
  else if (dtype == NFS_C64)
    e = nfs::matvec_launch_mask<float>(margs<float>(c, (const float2*)u, (float2*)Au, nullptr), mask);
  else
    return NFS_EINVAL;
  if (e != cudaSuccess) return cuda_fail(e, "nfs_matvec_passes");
  return NFS_OK;
}

extern "C" int nfs_apply_Br(nfs_ctx* c, const void* v, void* out) {
  if (!c || !v || !out || v == out) return NFS_EINVAL;
  return apply_Br(c, (const double2*)v, (double2*)out);
}

extern "C" int nfs_cg_solve(nfs_ctx* c, const void* b, void* x, nfs_solve_info* info) {
  if (!c || !b || !x || b == x) return NFS_EINVAL;
  const int r = solve(c, (const double2*)b, (double2*)x, false, info);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "nfs_cg_solve");
  return r;
}

extern "C" int nfs_eigs(nfs_ctx* c, int nev, double* omega, void* Y, nfs_eigs_info* info) {
  if (!c || !omega || nev <= 0 || nev >= c->N / 2) return NFS_EINVAL;
  const long long N = c->N;
  int m = c->opt.ncv > 0 ? c->opt.ncv : std::max(3 * nev, 2 * nev + 2);
  m = (int)std::min<long long>(m, N - 1);
  if (m <= nev + 1) return NFS_EINVAL;
  TRY(ensure_basis(c, m));
  TRY(ensure_scratch(c, lanczos_scratch_len(c->vcap)));
  const long long mv32_0 = c->mv32, mv64_0 = c->mv64;
  double2* V = c->V;
  double2* MV = c->MV;
  auto vec = [&](double2* base, int j) { return base + (long long)j * N; };
  const int nb = grid_blocks(N, 256);

  // starting vector, A_r-normalised
  nfs::k_random_fill<<<nb, 256, 0, c->stream>>>(vec(V, 0), N, c->opt.seed);
  CK(cudaGetLastError());
  TRY(matvec<double>(c, vec(V, 0), vec(MV, 0)));
  double nrm2;
  TRY(dot_re(c, vec(V, 0), vec(MV, 0), &nrm2));
  if (!(nrm2 > 0)) return NFS_EBREAKDOWN;
  nfs::k_scale<double2><<<nb, 256, 0, c->stream>>>(vec(V, 0), 1.0 / std::sqrt(nrm2), N);
  nfs::k_scale<double2><<<nb, 256, 0, c->stream>>>(vec(MV, 0), 1.0 / std::sqrt(nrm2), N);
  CK(cudaGetLastError());

  const int keep = std::min(m - 1, std::max(nev + 1, nev + (m - nev) / 2));
  std::vector<double> H((size_t)m * m, 0.0);
  int jstart = 0;
  double beta_last = 0.0;
  long long cg_total = 0;
  int steps = 0, restarts = 0, nconv = 0, status = NFS_OK;
  std::vector<double> theta, Z, coef, coef2;
  std::vector<int> order;
  double2* w = c->t64;    // new Krylov vector
  double2* Mw = c->t64b;  // A_r w
  for (;;) {
    for (int j = jstart; j < m; ++j) {
      // w = A_r^{-1} B_r v_j (CG); A_r w = B_r v_j
      TRY(apply_Br(c, vec(V, j), Mw));
      nfs_solve_info si{};
      const int rs = solve(c, Mw, w, true, &si);
      if (rs == NFS_EBREAKDOWN) return NFS_EBREAKDOWN;
      cg_total += si.iterations;
      ++steps;
      // classical Gram-Schmidt, twice, in the A_r inner product
      TRY(multi_dot(c, MV, j + 1, w, coef));
      TRY(multi_axpy(c, w, Mw, V, MV, j + 1, coef));
      TRY(multi_dot(c, MV, j + 1, w, coef2));
      TRY(multi_axpy(c, w, Mw, V, MV, j + 1, coef2));
      const double alpha = coef[2 * j] + coef2[2 * j];
      double bb;
      TRY(dot_re(c, w, Mw, &bb));
      if (!(bb > 0)) return NFS_EBREAKDOWN;
      const double beta = std::sqrt(bb);
      H[(size_t)j * m + j] = alpha;
      if (j + 1 < m) H[(size_t)(j + 1) * m + j] = H[(size_t)j * m + j + 1] = beta;
      beta_last = beta;
      nfs::k_scale<double2><<<nb, 256, 0, c->stream>>>(w, 1.0 / beta, N);
      nfs::k_scale<double2><<<nb, 256, 0, c->stream>>>(Mw, 1.0 / beta, N);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(vec(V, j + 1), w, N * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(vec(MV, j + 1), Mw, N * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    }
    // Rayleigh-Ritz on the projected matrix; theta = 1/omega, largest first
    jacobi_eig(m, H, theta, Z);
    order.resize(m);
    for (int i = 0; i < m; ++i) order[i] = m - 1 - i;  // descending theta
    nconv = 0;
    for (int i = 0; i < nev; ++i) {
      const int col = order[i];
      const double res = std::fabs(beta_last * Z[(size_t)(m - 1) * m + col]);
      if (res <= c->opt.eig_tol * std::fabs(theta[col])) ++nconv;
    }
    if (nconv == nev || restarts >= c->opt.max_restarts) {
      if (nconv < nev) status = NFS_ENOCONV;
      break;
    }
    // thick restart: keep the `keep` largest Ritz pairs
    std::vector<double> Ycm((size_t)m * keep);
    for (int i = 0; i < keep; ++i)
      for (int r = 0; r < m; ++r) Ycm[(size_t)i * m + r] = Z[(size_t)r * m + order[i]];
    TRY(rotate(c, V, m, Ycm, keep));
    TRY(rotate(c, MV, m, Ycm, keep));
    CK(cudaMemcpyAsync(vec(V, keep), vec(V, m), N * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(vec(MV, keep), vec(MV, m), N * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    std::fill(H.begin(), H.end(), 0.0);
    for (int i = 0; i < keep; ++i) {
      H[(size_t)i * m + i] = theta[order[i]];
      const double s = beta_last * Z[(size_t)(m - 1) * m + order[i]];
      H[(size_t)keep * m + i] = H[(size_t)i * m + keep] = s;
    }
    jstart = keep;
    ++restarts;
  }
  // results: omega ascending = theta descending (all wanted theta > 0)
  double maxres = 0.0;
  for (int i = 0; i < nev; ++i) {
    const int col = order[i];
    omega[i] = 1.0 / theta[col];
    maxres = std::max(maxres, std::fabs(beta_last * Z[(size_t)(m - 1) * m + col]) / std::fabs(theta[col]));
  }
  if (Y) {
    // Y[:, i] = V[0:m] z_i  (written through the rotation kernel into a copy)
    std::vector<double> Ycm((size_t)m * nev);
    for (int i = 0; i < nev; ++i)
      for (int r = 0; r < m; ++r) Ycm[(size_t)i * m + r] = Z[(size_t)r * m + order[i]];
    TRY(rotate(c, V, m, Ycm, nev));
    CK(cudaMemcpyAsync(Y, V, (size_t)nev * N * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  if (info) {
    info->lanczos_steps = steps;
    info->restarts = restarts;
    info->cg_iterations = cg_total;
    info->matvecs_c64 = c->mv32 - mv32_0;
    info->matvecs_c128 = c->mv64 - mv64_0;
    info->nconv = nconv;
    info->max_ritz_residual = maxres;
    info->status = status;
  }
  return status;
}

extern "C" int nfs_eig_grad(nfs_ctx* c, int m, const double* weights, const void* Yv, double* d_eps,
                            double* d_gamma) {
  if (!c || m <= 0 || !weights || !Yv) return NFS_EINVAL;
  if (c->has_mu) return NFS_EUNSUPPORTED;
  const long long n = c->n, N = c->N;
  if (d_eps) CK(cudaMemsetAsync(d_eps, 0, 3 * n * sizeof(double), c->stream));
  if (d_gamma) CK(cudaMemsetAsync(d_gamma, 0, c->gam_len * sizeof(double), c->stream));
  const double2* Y = (const double2*)Yv;
  for (int j = 0; j < m; ++j) {
    const double2* y = Y + (long long)j * N;
    TRY(apply_Br(c, y, c->t64));
    double yBy;
    TRY(dot_re(c, y, c->t64, &yBy));
    if (!(yBy != 0.0)) return NFS_EINVAL;
    const double scale = weights[j] / ((double)n * yBy);
    cudaError_t e = nfs::pass1_launch<double>(margs<double>(c, y, nullptr, nullptr));
    if (e != cudaSuccess) return cuda_fail(e, "grad pass 1");
    nfs::GradArgs g{};
    g.fld = (const double2*)c->fld; g.tw3 = c->tw64[2];
    g.inv_phi = c->mat64; g.gam = c->mat64 + 3 * n;
    g.kind = c->kind; g.ax_a = c->ax_a; g.ax_b = c->ax_b;
    g.n1 = c->n1; g.n2 = c->n2; g.n3 = c->n3;
    g.scale = scale; g.d_eps = d_eps; g.d_gamma = d_gamma; g.stream = c->stream;
    e = nfs::grad_launch(g);
    if (e != cudaSuccess) return cuda_fail(e, "grad launch");
  }
  CK(cudaStreamSynchronize(c->stream));
  return NFS_OK;
}
