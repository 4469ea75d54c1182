// libnfs C ABI: context setup, A_r and B_r products, CG (FP64 and mixed
// precision with FP64 refinement), thick-restart invert Lanczos on the
// HHPD-NFGEP, the eigenvalue gradient, and batches of independent problems.
// See include/nfs.h.
//
// A context holds P >= 1 problems that share one grid (different k-points
// and media).  Every kernel serves all P problems in one launch (the problem
// index is a grid dimension), and the solvers run the P problems in lock-step
// with per-problem scalars on the host; problems that have converged are
// masked out.  nfs_setup makes a context with P = 1; nfs_setup_batch groups
// a batch by grid into such contexts and drives each from its own host thread
// and stream, so different grid sizes overlap on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <map>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/nfs.h"
#include "blas_kernels.cuh"
#include "dfloat.cuh"
#include "host_eig.h"
#include "host_zeig.h"
#include "krylov.h"
#include "matvec.h"
#include "nfsep.h"

using nfs::CGState;
using nfs::kRedBlocks;
using nfs::kRedThreads;

namespace {
struct GraphEntry {
  const void* key[5];
  cudaGraphExec_t exec;
};
// A batch of GMRES steps as a replayable graph: steps j0 .. j0 + nsteps - 1
// of a cycle of length m, for one shift.
struct GmresGraph {
  int j0, nsteps, m;
  const void* V;
  const void* w;
  const void* scratch;
  double sigma_re, sigma_im;
  long long kernels;  // kernel launches one replay makes
  cudaGraphExec_t exec;
};
}  // namespace

struct nfs_ctx {
  int n1 = 0, n2 = 0, n3 = 0, nl = 0;
  long long n = 0, N = 0;  // voxels, 4n
  int P = 1;               // problems in this context
  double delta[3] = {0, 0, 0};
  nfs_options opt{};
  cudaStream_t stream = nullptr;  // caller's stream
  cudaStream_t work = nullptr;    // the library's own stream (CG and Lanczos; graph capture)
  cudaEvent_t ev = nullptr;
  int kind = 0, ax_a = 0, ax_b = 1;
  bool has_mu = false;
  long long gam_len = 0, mat_len = 0;
  // tables (per problem: stride nl) and twiddles (shared)
  double2* lam64 = nullptr;
  float2* lam32 = nullptr;
  double2* tw64[3] = {nullptr, nullptr, nullptr};
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  // material, per problem (stride mat_len): inv_phi [3n] | gam [3n or n] | inv_mu [3n]
  double* mat64 = nullptr;
  float* mat32 = nullptr;
  double2* basis64 = nullptr;  // per problem [6][n]: c and x of every voxel (complex128 products)
  // Bloch twist of T (eq. mtx_T), per problem (stride nl): the diagonals
  // D_l[j] = exp(i 2 pi k.a_l j / n_l), l = 1, 2, 3; and k.a_l itself
  double2* bloch64 = nullptr;
  std::vector<double> kd;
  // media outside the Assumption (nfs_setup_biiso): B^{-1} per voxel and
  // component as 2 x 2 blocks [4 * 3][n]; the Arnoldi and GMRES bases and the
  // device copy of rotation coefficients of the NFSEP eigensolve
  double2* binv64 = nullptr;
  double2* zv = nullptr;
  double2* gv = nullptr;
  double* zY = nullptr;
  int zv_cap = 0, gv_cap = 0;
  size_t zY_len = 0;
  // double-single copies of the tables, material and basis (mixed contexts:
  // the refinement residual products)
  nfs::dfc* lamdf = nullptr;
  nfs::dfc* twdf[3] = {nullptr, nullptr, nullptr};
  nfs::df* matdf = nullptr;
  nfs::dfc* basisdf = nullptr;
  // workspaces, per problem
  void* fld = nullptr;  // 6n complex128 each (complex64 uses 12n entries of it)
  double2 *x64 = nullptr, *r64 = nullptr, *p64 = nullptr, *Ap64 = nullptr, *t64 = nullptr, *t64b = nullptr;
  float2 *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *Ap32 = nullptr;
  float2* p32b = nullptr;  // second CG direction buffer when pass 1 cannot update in place
  CGState* st = nullptr;
  CGState* st_host = nullptr;  // pinned mirror of the scalar part
  // small per-problem arrays (device + pinned host): tolerances, scales, flags
  double* d_small = nullptr;
  double* h_small = nullptr;
  int* d_flags = nullptr;
  int* h_flags = nullptr;
  double* dscratch = nullptr;  // reductions
  size_t dscratch_len = 0;
  double* hscratch = nullptr;  // pinned
  size_t hscratch_len = 0;
  // Lanczos basis (FP64) and its complex64 shadows; problem stride vcap * N
  double2* V = nullptr;
  double2* MV = nullptr;
  float2* V32 = nullptr;
  float2* MV32 = nullptr;
  float2* MV32lo = nullptr;  // FP64 remainder of the MV32 shadow
  int vcap = 0;
  double* dY = nullptr;  // rotation coefficients
  int ncv_set = 0;       // basis size chosen by a batch for this context (0: own default)
  size_t dY_len = 0;
  std::vector<GraphEntry> graphs;
  std::vector<GmresGraph> gm_graphs;  // NFSEP inner-solve step batches
  long long bytes = 0;
  long long mv32 = 0, mv64 = 0;
  long long launches = 0;  // kernels this context has launched (graph nodes included)
  double sec_cg = 0.0;     // host wall time inside the CG iteration loops
  double sec_solve = 0.0;  // ... inside whole solves (CG + refinement residuals)
  double sec_ritz = 0.0;   // ... in the host projected eigensolves
  double sec_recur = 0.0, sec_orth = 0.0, sec_vec = 0.0;  // Lanczos phases
};

struct nfs_batch {
  std::vector<nfs_ctx*> classes;
  std::vector<std::pair<int, int>> where;  // problem -> (class, index in class)
};

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

thread_local char g_errbuf[256];

// Opt-in trace of the Lanczos steps on stderr (NFS_TRACE_LANCZOS set in the
// environment): per step alpha, beta^2 before and after the
// re-orthogonalisation, the measured loss and the CG status; read once.
bool trace_lanczos() {
  static const bool on = std::getenv("NFS_TRACE_LANCZOS") != nullptr;
  return on;
}

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_errbuf, sizeof(g_errbuf), "%s: %s", what, cudaGetErrorString(e));
  return NFS_ECUDA;
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);            \
  } while (0)

#define TRY(call)                 \
  do {                            \
    int r_ = (call);              \
    if (r_ != NFS_OK) return r_;  \
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

bool size_ok(int s) {
  switch (s) {
    case 8: case 12: case 16: case 24: case 32: case 48: case 64: case 96: case 128: return true;
    default: return false;
  }
}

int grid_blocks(long long N, int threads) {
  long long b = (N + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 16));
}

// --- matvec -------------------------------------------------------------

nfs::BatchStrides strides(const nfs_ctx* c, long long sfld) {
  nfs::BatchStrides b;
  b.su = c->N;
  b.sfld = sfld;
  b.smat = c->mat_len;
  b.sstate = nfs::kStateDoubles;
  b.slam = c->nl;
  b.sskip = nfs::kStateInts;
  return b;
}

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
  a.basis = c->basis64;
  a.P = c->P;
  a.bs = strides(c, 6 * c->n);
  a.bs.sbasis = 6 * c->n;
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
  a.P = c->P;
  a.bs = strides(c, 12 * c->n);  // the complex128-sized workspace holds 12 n complex64 per problem
  return a;
}

template <>
nfs::MatvecArgs<nfs::df> margs<nfs::df>(nfs_ctx* c, const nfs::dfc* u, nfs::dfc* Au, const int* skip) {
  nfs::MatvecArgs<nfs::df> a{};
  a.u = u; a.Au = Au; a.fld = (nfs::dfc*)c->fld; a.lam = c->lamdf;
  a.tw1 = c->twdf[0]; a.tw2 = c->twdf[1]; a.tw3 = c->twdf[2];
  a.inv_phi = c->matdf; a.gam = c->matdf + 3 * c->n; a.inv_mu = c->has_mu ? c->matdf + 3 * c->n + c->gam_len : nullptr;
  a.kind = c->kind; a.ax_a = c->ax_a; a.ax_b = c->ax_b;
  a.n1 = c->n1; a.n2 = c->n2; a.n3 = c->n3; a.alpha = nfs::df(c->opt.alpha); a.beta = nfs::df(c->opt.beta);
  a.skip = skip; a.stream = c->stream;
  a.basis = c->basisdf;
  a.P = c->P;
  a.bs = strides(c, 6 * c->n);
  a.bs.sbasis = 6 * c->n;
  return a;
}

// P products (problem p's vectors at u + p N); skip (optional): problem p is
// skipped when skip[p * sskip] is nonzero.
template <typename R>
int matvec(nfs_ctx* c, cudaStream_t s, const nfs::cplx<R>* u, nfs::cplx<R>* Au, const int* skip = nullptr,
           int sskip = 0) {
  nfs::MatvecArgs<R> a = margs<R>(c, u, Au, skip);
  a.stream = s;
  a.bs.sskip = sskip;
  cudaError_t e = nfs::matvec_launch<R>(a);
  if (e != cudaSuccess) return cuda_fail(e, "matvec launch");
  c->launches += nfs::product_kernels<R>(c->n1);
  if (sizeof(nfs::cplx<R>) == 8) c->mv32 += c->P; else c->mv64 += c->P;
  return NFS_OK;
}

// FP64-accuracy products of complex128 vectors through the double-single
// product (mixed contexts): u is converted into the free CG direction buffer
// p64, the result is written into out and converted there in place.
int matvec_refine(nfs_ctx* c, cudaStream_t s, const double2* u, double2* out, const int* skip, int sskip) {
  const long long reals = 2 * c->P * c->N;
  nfs::dfc* uin = reinterpret_cast<nfs::dfc*>(c->p64);
  nfs::dfc* res = reinterpret_cast<nfs::dfc*>(out);
  CK(nfs::double_to_df(reinterpret_cast<const double*>(u), reinterpret_cast<nfs::df*>(uin), reals, s));
  TRY(matvec<nfs::df>(c, s, uin, res, skip, sskip));
  CK(nfs::df_to_double(reinterpret_cast<const nfs::df*>(res), reinterpret_cast<double*>(out), reals, s));
  c->launches += 2;
  return NFS_OK;
}

// --- scratch ---------------------------------------------------------------

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

// Blocks per problem of the reductions over P problems' vectors of length N.
// Never more blocks than the vector has threads' worth of elements (empty
// blocks add exact zeros: a single problem's sums are the same at any larger
// count); for batches, fewer, with at least 32 elements per thread, as long
// as all problems together still have kRedBlocks blocks.  Each block ends in
// FP64 block sums, which GB300 retires at about one warp instruction per 17
// SM cycles: a full grid per problem over the short vectors of a batch of
// small grids made those epilogues, not the data, the cost of a reduction.
int red_blocks(long long N, int P) {
  long long nb = std::min<long long>(kRedBlocks, (N + kRedThreads - 1) / kRedThreads);
  if (P > 1) {
    const long long per32 = (N + (long long)kRedThreads * 32 - 1) / ((long long)kRedThreads * 32);
    nb = std::min(nb, std::max<long long>(per32, (kRedBlocks + P - 1) / P));
  }
  return (int)std::max<long long>(1, nb);
}

// Re(x_p^* y_p) for every problem, on the host
template <typename C>
int dots_re(nfs_ctx* c, cudaStream_t s, const C* x, const C* y, std::vector<double>& out) {
  const int nb = red_blocks(c->N, c->P);
  nfs::k_dot_re<C><<<dim3(nb, c->P), kRedThreads, 0, s>>>(x, y, c->N, c->dscratch, nb, nullptr, 0);
  CK(cudaGetLastError());
  c->launches += 1;
  CK(cudaMemcpyAsync(c->hscratch, c->dscratch, (size_t)nb * c->P * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out.assign(c->P, 0.0);
  for (int p = 0; p < c->P; ++p) {
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += c->hscratch[(size_t)p * nb + i];
    out[p] = t;
  }
  return NFS_OK;
}

// Layout of d_small (doubles): [0, P) tolerances, [P, 2P) and [2P, 3P) scales;
// of d_flags (ints): [0, P) active problems, [P, 2P) a second mask, [2P, 4P)
// the skip masks of the two refinement products.
constexpr int kSmallSlots = 3;
constexpr int kFlagSlots = 4;

// upload v to c->d_small + off through the pinned mirror
int put_small(nfs_ctx* c, cudaStream_t s, int off, const std::vector<double>& v) {
  std::memcpy(c->h_small + off, v.data(), v.size() * sizeof(double));
  CK(cudaMemcpyAsync(c->d_small + off, c->h_small + off, v.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  return NFS_OK;
}

int put_flags(nfs_ctx* c, cudaStream_t s, int off, const std::vector<int>& v) {
  std::memcpy(c->h_flags + off, v.data(), v.size() * sizeof(int));
  CK(cudaMemcpyAsync(c->d_flags + off, c->h_flags + off, v.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  return NFS_OK;
}

// --- CG ---------------------------------------------------------------------

// CG iterations per captured chunk (even); the host reads the done flags
// between chunks, and iterations launched after convergence return at once
#ifndef NFS_CG_CHUNK
#define NFS_CG_CHUNK 8
#endif
constexpr int kCgChunk = NFS_CG_CHUNK;

// Enqueue kCgChunk iterations for all problems: pass 1 (which first forms
// p = r + beta p), passes 2 and 3 (pass 2 also emits the p^* A p partials,
// from the real-space fields) and the x/r update (which forms alpha, and in
// its last block beta).
template <typename R>
cudaError_t enqueue_cg_chunk(nfs_ctx* c, cudaStream_t s, nfs::cplx<R>* x, nfs::cplx<R>* r, nfs::cplx<R>* p,
                             nfs::cplx<R>* Ap) {
  using C = nfs::cplx<R>;
  nfs::MatvecArgs<R> a = margs<R>(c, p, Ap, &c->st->done);
  a.stream = s;
  a.cg_r = r;
  a.cg_beta = &c->st->beta;
  a.dot_part = c->st->part_a;
  // kernels that cannot form p = r + beta p in place alternate between p and
  // a second buffer (kCgChunk is even: p holds the direction after a chunk)
  C* p2 = nullptr;
  if (sizeof(R) == 4 && nfs::cg_needs_p_out<R>(c->n1)) p2 = reinterpret_cast<C*>(c->p32b);
  static_assert(kCgChunk % 2 == 0, "the direction must end a chunk in p");
  // where pass 3 can take the x/r step itself, no update kernel runs and A p
  // is never stored
  const bool fused = nfs::cg_fusable<R>(c->n1);
  for (int i = 0; i < kCgChunk; ++i) {
    C* pn = p;
    if (p2 != nullptr) {
      a.u = (i % 2 == 0) ? p : p2;
      pn = (i % 2 == 0) ? p2 : p;
      a.p_out = pn;
    }
    if (fused) {
      a.cg.x = x;
      a.cg.r = r;
      a.cg.p = pn;
      a.cg.st = c->st;
    }
    cudaError_t e = nfs::matvec_launch<R>(a);
    if (e != cudaSuccess) return e;
    if (!fused) {
      nfs::k_cg_update_xr<C><<<dim3(nfs::kUpdBlocks, c->P), nfs::kUpdThreads, 0, s>>>(x, r, pn, Ap, c->N, c->st);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// The chunk as a CUDA graph, captured once per (precision, buffers) on the
// context's work stream and replayed: one launch per chunk instead of
// 4 kCgChunk kernel launches.
template <typename R>
int cg_chunk_graph(nfs_ctx* c, nfs::cplx<R>* x, nfs::cplx<R>* r, nfs::cplx<R>* p, nfs::cplx<R>* Ap,
                   cudaGraphExec_t* out) {
  const void* key[5] = {x, r, p, Ap, (const void*)(uintptr_t)sizeof(R)};
  for (const GraphEntry& g : c->graphs)
    if (std::equal(key, key + 5, g.key)) {
      *out = g.exec;
      return NFS_OK;
    }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(c->work, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_cg_chunk<R>(c, c->work, x, r, p, Ap);
  cudaError_t e2 = cudaStreamEndCapture(c->work, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e, "cg capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  GraphEntry g;
  std::copy(key, key + 5, g.key);
  g.exec = exec;
  c->graphs.push_back(g);
  *out = exec;
  return NFS_OK;
}

// CG from the state r = b - A x (already formed) for every problem, on the
// work stream; tol2 the absolute thresholds on r^* r (+inf skips a problem).
// Iterations run in graph-replayed chunks; every kernel returns at once after
// its problem's device `done` flag is set, and the host reads the flags
// between chunks.
template <typename R>
int cg_run(nfs_ctx* c, nfs::cplx<R>* x, nfs::cplx<R>* r, nfs::cplx<R>* p, nfs::cplx<R>* Ap,
           const std::vector<double>& tol2, int maxit, std::vector<int>& iters, std::vector<int>& status) {
  using C = nfs::cplx<R>;
  cudaStream_t s = c->work;
  CK(cudaStreamSynchronize(s));  // earlier work is not the loop's
  const double t0 = now_s();
  CK(cudaMemsetAsync(p, 0, c->P * c->N * sizeof(C), s));  // with beta = 0 the first pass 1 sets p = r
  const int nb = red_blocks(c->N, c->P);
  nfs::k_dot_re<C><<<dim3(nb, c->P), kRedThreads, 0, s>>>(r, r, c->N, c->st->part_a, nfs::kStateDoubles, nullptr, 0);
  TRY(put_small(c, s, 0, tol2));
  nfs::k_cg_init<<<c->P, kRedThreads, 0, s>>>(c->st, c->d_small, maxit,
                                               nfs::matvec_dot_partials<R>(c->n1, c->n2, c->n3), nb);
  CK(cudaGetLastError());
  c->launches += 2;
  cudaGraphExec_t exec = nullptr;
  TRY(cg_chunk_graph<R>(c, x, r, p, Ap, &exec));
  const size_t head = offsetof(CGState, part_a);
  for (;;) {
    CK(cudaGraphLaunch(exec, s));
    c->launches += (nfs::product_kernels<R>(c->n1) + (nfs::cg_fusable<R>(c->n1) ? 0 : 1)) * kCgChunk;
    CK(cudaMemcpy2DAsync(c->st_host, sizeof(CGState), c->st, sizeof(CGState), head, c->P, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool all = true;
    for (int q = 0; q < c->P; ++q) all = all && c->st_host[q].done;
    if (all) break;
  }
  iters.resize(c->P);
  status.resize(c->P);
  for (int q = 0; q < c->P; ++q) {
    iters[q] = c->st_host[q].it;
    status[q] = c->st_host[q].status;
    // one product per iteration that ran (launches after convergence are empty)
    if (sizeof(R) == 4) c->mv32 += iters[q]; else c->mv64 += iters[q];
  }
  c->sec_cg += now_s() - t0;
  return NFS_OK;
}

int sub64(nfs_ctx* c, cudaStream_t s, const double2* a, const double2* b, double2* y) {
  const long long tot = c->P * c->N;
  nfs::k_sub<double2><<<grid_blocks(tot, 256), 256, 0, s>>>(a, b, y, tot);
  CK(cudaGetLastError());
  c->launches += 1;
  return NFS_OK;
}

// Solve A_r x_p = b_p for every problem p with active[p] (b, x: P x N, on the
// work stream).  FP64 contexts run complex128 CG; MIXED contexts run complex64
// CG inside FP64 iterative refinement (the residual r = b - A_r x with the
// complex128 product, scaled to unit norm, demoted; x += |r| d).
struct SolveOut {
  std::vector<int> iters, refines, status;
  std::vector<double> relres;
};

int solve(nfs_ctx* c, const double2* b, double2* x, bool x_zero, const std::vector<int>& active, SolveOut& so) {
  cudaStream_t s = c->work;
  const int P = c->P;
  const long long tot = P * c->N;
  std::vector<double> bb;
  TRY(dots_re(c, s, b, b, bb));
  so.iters.assign(P, 0);
  so.refines.assign(P, 0);
  so.status.assign(P, NFS_OK);
  so.relres.assign(P, 0.0);
  if (x_zero) {
    CK(cudaMemsetAsync(x, 0, tot * sizeof(double2), s));
    CK(cudaMemcpyAsync(c->r64, b, tot * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  } else {
    TRY(matvec<double>(c, s, x, c->Ap64));
    TRY(sub64(c, s, b, c->Ap64, c->r64));
  }
  const double tol = c->opt.cg_tol;
  std::vector<int> need(P);
  for (int q = 0; q < P; ++q) need[q] = active[q] && bb[q] > 0.0;
  if (c->opt.precision != NFS_PREC_MIXED) {
    std::vector<double> tol2(P);
    for (int q = 0; q < P; ++q) tol2[q] = need[q] ? tol * tol * bb[q] : INFINITY;
    std::vector<int> it, st;
    TRY(cg_run<double>(c, x, c->r64, c->p64, c->Ap64, tol2, c->opt.cg_maxit, it, st));
    for (int q = 0; q < P; ++q) {
      if (!need[q]) continue;
      so.iters[q] = it[q];
      so.status[q] = st[q];
      so.relres[q] = std::sqrt(std::max(c->st_host[q].rr, 0.0) / bb[q]);
    }
    return NFS_OK;
  }
  // mixed precision.  Round k: d = A32^{-1} (r_k / |r_k|) by complex64 CG,
  // x += |r_k| d, then the next residual.  While the correction is of the
  // size of x (|r_k| large) the residual needs the complex128 product,
  // r = b - A x.  Once |r_k| <= kCheapRefine * tol * |b| it is updated as
  // r -= |r_k| A32 d with the complex64 product of the correction: that
  // product's relative error (~5e-7) then moves r by at most ~1% of the
  // tolerance.  The inner tolerance is inner_tol, or looser where the
  // remaining reduction tol |b| / |r_k| asks for less.
  constexpr double kCheapRefine = 2.5e4;
  const int nb = grid_blocks(tot, 256);
  std::vector<double> rr;
  std::vector<int> live(need);
  for (;;) {
    TRY(dots_re(c, s, c->r64, c->r64, rr));
    bool any = false, any64 = false, any32 = false;
    std::vector<double> inv(P, 0.0), nrm(P, 0.0), itol2(P, INFINITY);
    std::vector<int> skip(P, 1), skip64(P, 1), skip32(P, 1);
    for (int q = 0; q < P; ++q) {
      if (!live[q]) continue;
      so.relres[q] = std::sqrt(std::max(rr[q], 0.0) / bb[q]);
      if (!(rr[q] == rr[q])) { so.status[q] = NFS_EBREAKDOWN; live[q] = 0; continue; }
      if (rr[q] <= tol * tol * bb[q]) { live[q] = 0; continue; }
      if (so.refines[q] >= c->opt.max_refine) { so.status[q] = NFS_ENOCONV; live[q] = 0; continue; }
      any = true;
      nrm[q] = std::sqrt(rr[q]);
      inv[q] = 1.0 / nrm[q];
      const double need_red = 0.3 * tol * std::sqrt(bb[q]) / nrm[q];
      const double itol = std::max(c->opt.inner_tol, std::min(need_red, 0.1));
      itol2[q] = itol * itol;
      skip[q] = 0;
      if (nrm[q] <= kCheapRefine * tol * std::sqrt(bb[q])) {
        skip32[q] = 0;
        any32 = true;
      } else {
        skip64[q] = 0;
        any64 = true;
      }
    }
    if (!any) break;
    TRY(put_small(c, s, P, inv));
    nfs::k_demote<<<nb, 256, 0, s>>>(c->r64, c->d_small + P, c->r32, c->N, tot);
    CK(cudaGetLastError());
    c->launches += 1;
    CK(cudaMemsetAsync(c->x32, 0, tot * sizeof(float2), s));
    std::vector<int> it, st;
    TRY(cg_run<float>(c, c->x32, c->r32, c->p32, c->Ap32, itol2, c->opt.cg_maxit, it, st));
    TRY(put_small(c, s, 2 * P, nrm));
    nfs::k_axpy_promote<<<nb, 256, 0, s>>>(x, c->d_small + 2 * P, c->x32, c->N, tot);
    CK(cudaGetLastError());
    c->launches += 1;
    // next residual: complex128 product of x, or complex64 product of d
    TRY(put_flags(c, s, 2 * P, skip64));
    TRY(put_flags(c, s, 3 * P, skip32));
    if (any64) TRY(matvec_refine(c, s, x, c->Ap64, c->d_flags + 2 * P, 1));
    if (any32) TRY(matvec<float>(c, s, c->x32, c->Ap32, c->d_flags + 3 * P, 1));
    nfs::k_refine_residual<<<nb, 256, 0, s>>>(c->r64, b, c->Ap64, c->Ap32, c->d_small + 2 * P, c->d_flags + 2 * P,
                                              c->d_flags + 3 * P, c->N, tot);
    CK(cudaGetLastError());
    c->launches += 1;
    for (int q = 0; q < P; ++q) {
      if (skip[q]) continue;
      so.iters[q] += it[q];
      so.refines[q] += 1;
      if (st[q] == NFS_EBREAKDOWN) { so.status[q] = NFS_EBREAKDOWN; live[q] = 0; }
    }
  }
  return NFS_OK;
}

// --- Lanczos helpers -------------------------------------------------------

// Lanczos scratch layout in dscratch (doubles), mcap the basis capacity:
//   [0, P * kRedBlocks * 2 * mcap)   per-block partial dots
//   then P * 2 * mcap                finished dots
//   then P * 2 * mcap                coefficients for the update
size_t lanczos_scratch_len(int P, int mcap) {
  return (size_t)P * kRedBlocks * 2 * mcap + 4 * (size_t)P * mcap + 64;
}
size_t off_fin(const nfs_ctx* c) { return (size_t)c->P * kRedBlocks * 2 * c->vcap; }
size_t off_coef(const nfs_ctx* c) { return off_fin(c) + (size_t)2 * c->P * c->vcap; }

// Per-problem complex inner products of w_p with basis vectors [j0, j0 + m) of
// Vbase (V or MV, FP64) -> out[p * 2m + 2i + {0,1}] on the host; problems with
// a zero flag in d_active are skipped.
int multi_dot(nfs_ctx* c, const double2* Vbase, int j0, int m, const double2* w, std::vector<double>& out,
              const int* d_active) {
  cudaStream_t s = c->work;
  const long long vstride = (long long)c->vcap * c->N;
  double* part = c->dscratch;
  double* fin = c->dscratch + off_fin(c);
  const int nb = red_blocks(c->N, c->P);
  nfs::k_multi_dot<kRedThreads><<<dim3(nb, c->P), kRedThreads, 0, s>>>(Vbase + (long long)j0 * c->N, vstride,
                                                                              m, w, c->N, part, d_active);
  nfs::k_multi_dot_finish<<<dim3(m, c->P), kRedThreads, 0, s>>>(part, m, nb, fin, d_active);
  CK(cudaGetLastError());
  c->launches += 2;
  CK(cudaMemcpyAsync(c->hscratch, fin, (size_t)c->P * m * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out.assign(c->hscratch, c->hscratch + (size_t)c->P * 2 * m);
  return NFS_OK;
}

// w_p -= V_p[j0 : j0 + m] coef_p ; Mw_p -= MV_p[j0 : j0 + m] coef_p
int multi_axpy(nfs_ctx* c, double2* w, double2* Mw, int j0, int m, const std::vector<double>& coef,
               const int* d_active) {
  cudaStream_t s = c->work;
  const long long vstride = (long long)c->vcap * c->N;
  double* dcoef = c->dscratch + off_coef(c);
  std::memcpy(c->hscratch, coef.data(), coef.size() * sizeof(double));
  CK(cudaMemcpyAsync(dcoef, c->hscratch, coef.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  nfs::k_multi_axpy<<<dim3(grid_blocks(c->N, 256), c->P), 256, 0, s>>>(
      w, Mw, c->V + (long long)j0 * c->N, c->MV + (long long)j0 * c->N, vstride, dcoef, m, c->N, d_active);
  CK(cudaGetLastError());
  c->launches += 1;
  CK(cudaStreamSynchronize(s));  // the pinned staging buffer is reused next
  return NFS_OK;
}

// d_p = MV_p[0:m]^* w_p, exact to ~1e-14 of the terms, from the split FP32
// shadows of MV on the FP32 units (orthogonality monitor and coefficients)
int exact_dots(nfs_ctx* c, int m, const double2* w, std::vector<double>& out, const int* d_active) {
  cudaStream_t s = c->work;
  const long long vstride = (long long)c->vcap * c->N;
  // basis vectors per block: each block streams its slice of w once per G
  // vectors, so a larger G re-reads w less often, but each vector costs a
  // thread six accumulator registers; measured on GB300 at 96^3 (headline
  // orthogonalisation time): G = 2 0.309 s, 4 0.343 s, 8 0.53 s, 16 0.91 s
#ifndef NFS_EXACT_G
#define NFS_EXACT_G 2
#endif
  constexpr int G = NFS_EXACT_G;
  double* part = c->dscratch;
  double* fin = c->dscratch + off_fin(c);
  // w split once into floats (the CG work vectors x32 / r32 are free here)
  float2* whi = c->x32 ? c->x32 : reinterpret_cast<float2*>(c->Ap64);
  float2* wlo = c->x32 ? c->r32 : reinterpret_cast<float2*>(c->Ap64) + c->P * c->N;
  nfs::k_split_hi_lo<<<grid_blocks(c->P * c->N, 256), 256, 0, s>>>(w, whi, wlo, c->P * c->N);
  const int nb = red_blocks(c->N, c->P);
  nfs::k_exact_dots<G><<<dim3(nb, (m + G - 1) / G, c->P), kRedThreads, 0, s>>>(c->MV32, c->MV32lo, vstride, m,
                                                                                       whi, wlo, c->N, part, d_active);
  nfs::k_dots_finish<<<dim3(m, c->P), kRedThreads, 0, s>>>(part, m, nb, fin, d_active);
  CK(cudaGetLastError());
  c->launches += 3;
  CK(cudaMemcpyAsync(c->hscratch, fin, (size_t)c->P * m * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out.assign(c->hscratch, c->hscratch + (size_t)c->P * 2 * m);
  return NFS_OK;
}

int refresh_shadows(nfs_ctx* c, int first, int count) {
  const long long vstride = (long long)c->vcap * c->N;
  const long long len = (long long)count * c->N;
  const long long off = (long long)first * c->N;
  nfs::k_refresh_shadows<<<grid_blocks(len * c->P, 256), 256, 0, c->work>>>(
      c->V + off, c->MV + off, c->V32 + off, c->MV32 + off, c->MV32lo + off, vstride, len, c->P);
  CK(cudaGetLastError());
  c->launches += 1;
  return NFS_OK;
}

int ensure_basis(nfs_ctx* c, int m) {
  if (c->vcap >= m + 1) return NFS_OK;
  void* olds[] = {c->V, c->MV, c->V32, c->MV32, c->MV32lo};
  for (void* p : olds)
    if (p) cudaFree(p);
  c->bytes -= (long long)c->P * c->vcap * c->N * (16 + 16 + 8 + 8 + 8);
  c->V = c->MV = nullptr;
  c->V32 = c->MV32 = c->MV32lo = nullptr;
  c->vcap = 0;
  const size_t len = (size_t)c->P * (m + 1) * c->N;
  TRY(dalloc(c, &c->V, len));
  TRY(dalloc(c, &c->MV, len));
  TRY(dalloc(c, &c->V32, len));
  TRY(dalloc(c, &c->MV32, len));
  TRY(dalloc(c, &c->MV32lo, len));
  c->vcap = m + 1;
  return NFS_OK;
}

// V_p[0:k] = V_p[0:m] Y_p for every problem flagged in d_active (Y: P blocks
// of m x k, column-major); base is V or MV.
int rotate(nfs_ctx* c, double2* base, int m, const std::vector<double>& Y, int k, const int* d_active) {
  // Y as (hi, lo) float pairs (the kernel works in double-single); one float
  // pair has the size of one double, so dY holds them
  const size_t need = (size_t)c->P * m * k;
  if (c->dY_len < need) {
    if (c->dY) cudaFree(c->dY);
    c->dY = nullptr;
    TRY(dalloc(c, &c->dY, need));
    c->dY_len = need;
  }
  std::vector<float> yhl(2 * need);
  for (size_t i = 0; i < need; ++i) {
    const float h = (float)Y[i];
    yhl[2 * i] = h;
    yhl[2 * i + 1] = (float)(Y[i] - (double)h);
  }
  CK(cudaMemcpyAsync(c->dY, yhl.data(), need * sizeof(double), cudaMemcpyHostToDevice, c->work));
  // a tile of TE elements of all m vectors in shared memory: 32 while that
  // fits in 200 KB, else narrower; CPT output columns per thread (measured at
  // 96^3 with thick restarts, ncv 60: CPT 2 2.222 s, 4 2.241 s, 8 2.37 s)
#ifndef NFS_ROT_CPT
#define NFS_ROT_CPT 2
#endif
  constexpr int CPT = NFS_ROT_CPT;
  const float2* yhl_d = reinterpret_cast<const float2*>(c->dY);
  auto launch = [&](auto te) -> cudaError_t {
    constexpr int TE = decltype(te)::value;
    const size_t smem = (size_t)m * TE * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(nfs::k_rotate_basis<TE, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    nfs::k_rotate_basis<TE, CPT><<<dim3(grid_blocks((c->N + TE - 1) / TE, 1), c->P), 256, smem, c->work>>>(
        base, (long long)c->vcap * c->N, m, yhl_d, k, c->N, d_active);
    return cudaGetLastError();
  };
  const size_t row = (size_t)m * sizeof(float4);
  if (row * 32 <= 200 * 1024)
    CK(launch(std::integral_constant<int, 32>{}));
  else if (row * 16 <= 200 * 1024)
    CK(launch(std::integral_constant<int, 16>{}));
  else
    CK(launch(std::integral_constant<int, 8>{}));
  c->launches += 1;
  CK(cudaStreamSynchronize(c->work));  // the host copy of Y is released next
  return NFS_OK;
}

// B_r applied to basis vector j of every problem -> out (P x N); t64 is used
// to gather the vectors contiguously
int apply_Br_basis(nfs_ctx* c, int j, double2* out) {
  // B_r of basis column j of every problem, read in place (stride vcap N)
  const long long vstride = (long long)c->vcap * c->N;
  nfs::k_apply_Br<<<grid_blocks(c->n * c->P, 256), 256, 0, c->work>>>(c->V + (long long)j * c->N, out, c->lam64,
                                                                      c->n1, c->n2, c->n3, c->P, vstride);
  CK(cudaGetLastError());
  c->launches += 1;
  return NFS_OK;
}

// Device bytes per basis vector of a context: V, A_rV (complex128), their
// complex64 shadows and the remainder of the A_rV shadow.
double basis_bytes_per_vector(const nfs_ctx* c) { return (double)c->P * c->N * (16 + 16 + 8 + 8 + 8); }

int wanted_ncv(int nev) { return std::max(std::max(3 * nev, 2 * nev + 2), std::min(12 * nev, 320)); }

// Default basis size: generous (device memory is plentiful and restarts cost
// FP64 basis rotations and accuracy), a fixed function of nev: the same
// basis, the same iterates and the same speed whatever else holds the GPU.
// NFS_ENOMEM when it does not fit (set opt.ncv smaller, e.g. the paper's
// 3 nev).
int default_ncv(nfs_ctx* c, int nev) {
  if (c->ncv_set > 0) return c->ncv_set;
  return wanted_ncv(nev);
}

// Rayleigh-Ritz over the nev Ritz vectors of problem p (basis positions
// 0..nev-1 after a rotation): the pencil H z = theta G z with
// H = Y^* B_r Y and G = Y^* A_r Y (A_r Y from fresh products), formed with
// FP64 inner products and solved on the host (Cholesky of G, Schur form of the
// Hermitian L^-1 H L^-*).  Copies of a degenerate eigenvalue found by
// deflation checks were each converged against locked vectors that are only
// accurate to eig_tol, so their eigenvalues carry a first-order error; the
// Rayleigh quotients on the span of all nev vectors are accurate to second
// order.  theta: ascending order of omega = 1/theta on return; z: the
// row-major nev x nev complex coefficients (interleaved re, im), columns in
// that order.  flags: a device mask with problem p alone set.
int final_rayleigh_ritz(nfs_ctx* c, int p, int nev, const int* flags, std::vector<double>& theta,
                        std::vector<double>& z, int kout = -1) {
  using cplxd = std::complex<double>;
  const long long N = c->N, vstride = (long long)c->vcap * N;
  if (kout < 0) kout = nev;
  std::vector<cplxd> H((size_t)nev * nev), G((size_t)nev * nev);
  std::vector<double> d;
  // A_r y_i from fresh products (complex128, or double-single in mixed
  // contexts) of problem p alone
  std::vector<int> skip(c->P, 1);
  skip[p] = 0;
  TRY(put_flags(c, c->work, 2 * c->P, skip));
  const int* d_skip = c->d_flags + 2 * c->P;
  for (int i = 0; i < nev; ++i) {
    TRY(apply_Br_basis(c, i, c->t64));  // B_r y_i (every problem; p's is used)
    TRY(multi_dot(c, c->V, 0, nev, c->t64, d, flags));
    for (int j = 0; j < nev; ++j) H[(size_t)j * nev + i] = cplxd(d[(size_t)p * 2 * nev + 2 * j], d[(size_t)p * 2 * nev + 2 * j + 1]);
    CK(cudaMemcpyAsync(c->t64 + (long long)p * N, c->V + p * vstride + (long long)i * N, N * sizeof(double2),
                       cudaMemcpyDeviceToDevice, c->work));
    if (c->lamdf)
      TRY(matvec_refine(c, c->work, c->t64, c->t64b, d_skip, 1));
    else
      TRY(matvec<double>(c, c->work, c->t64, c->t64b, d_skip, 1));
    TRY(multi_dot(c, c->V, 0, nev, c->t64b, d, flags));
    for (int j = 0; j < nev; ++j) G[(size_t)j * nev + i] = cplxd(d[(size_t)p * 2 * nev + 2 * j], d[(size_t)p * 2 * nev + 2 * j + 1]);
  }
  // symmetrise (the inner products are exact only to rounding)
  for (int i = 0; i < nev; ++i)
    for (int j = 0; j <= i; ++j) {
      const cplxd h = 0.5 * (H[(size_t)i * nev + j] + std::conj(H[(size_t)j * nev + i]));
      const cplxd g = 0.5 * (G[(size_t)i * nev + j] + std::conj(G[(size_t)j * nev + i]));
      H[(size_t)i * nev + j] = h;
      H[(size_t)j * nev + i] = std::conj(h);
      G[(size_t)i * nev + j] = g;
      G[(size_t)j * nev + i] = std::conj(g);
    }
  // G = L L^*
  std::vector<cplxd> L((size_t)nev * nev, 0.0);
  for (int j = 0; j < nev; ++j) {
    double dj = G[(size_t)j * nev + j].real();
    for (int q = 0; q < j; ++q) dj -= std::norm(L[(size_t)j * nev + q]);
    if (!(dj > 0)) {
      if (trace_lanczos())
        std::fprintf(stderr, "nfs rayleigh-ritz: problem %d, Gram matrix of %d vectors not positive at %d (%.3e)\n", p,
                     nev, j, dj);
      return NFS_EBREAKDOWN;
    }
    const double ljj = std::sqrt(dj);
    L[(size_t)j * nev + j] = ljj;
    for (int i = j + 1; i < nev; ++i) {
      cplxd v = G[(size_t)i * nev + j];
      for (int q = 0; q < j; ++q) v -= L[(size_t)i * nev + q] * std::conj(L[(size_t)j * nev + q]);
      L[(size_t)i * nev + j] = v / ljj;
    }
  }
  // M = L^-1 H L^-*: forward substitution on the columns of H, then on the
  // columns of (L^-1 H)^*
  auto lsolve = [&](std::vector<cplxd>& X) {  // X <- L^-1 X, X row-major nev x nev
    for (int col = 0; col < nev; ++col)
      for (int i = 0; i < nev; ++i) {
        cplxd v = X[(size_t)i * nev + col];
        for (int q = 0; q < i; ++q) v -= L[(size_t)i * nev + q] * X[(size_t)q * nev + col];
        X[(size_t)i * nev + col] = v / L[(size_t)i * nev + i];
      }
  };
  std::vector<cplxd> M = H;
  lsolve(M);
  std::vector<cplxd> Mh((size_t)nev * nev);
  for (int i = 0; i < nev; ++i)
    for (int j = 0; j < nev; ++j) Mh[(size_t)i * nev + j] = std::conj(M[(size_t)j * nev + i]);
  lsolve(Mh);  // = L^-1 (L^-1 H)^* = (L^-1 H L^-*)^* = L^-1 H L^-* (Hermitian)
  std::vector<cplxd> Q;
  if (!nfs::host::complex_schur(nev, Mh, Q)) return NFS_EBREAKDOWN;
  // eigenvalues on the (real) diagonal; order by theta descending = omega ascending
  std::vector<int> ord(nev);
  for (int i = 0; i < nev; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(),
            [&](int a, int b) { return Mh[(size_t)a * nev + a].real() > Mh[(size_t)b * nev + b].real(); });
  theta.assign(kout, 0.0);
  z.assign((size_t)2 * nev * kout, 0.0);
  // z = L^-* Q: back substitution with L^* on each column of Q
  for (int o = 0; o < kout; ++o) {
    const int col = ord[o];
    theta[o] = Mh[(size_t)col * nev + col].real();
    std::vector<cplxd> x(nev);
    for (int i = nev - 1; i >= 0; --i) {
      cplxd v = Q[(size_t)i * nev + col];
      for (int q = i + 1; q < nev; ++q) v -= std::conj(L[(size_t)q * nev + i]) * x[q];
      x[i] = v / L[(size_t)i * nev + i];
    }
    for (int r = 0; r < nev; ++r) {
      z[2 * ((size_t)r * kout + o)] = x[r].real();
      z[2 * ((size_t)r * kout + o) + 1] = x[r].imag();
    }
  }
  return NFS_OK;
}

// Complex rotation V_p[0:k] = V_p[0:q] z (z: q x k row-major, interleaved) of
// problem p's V and MV through the device copy of z.
int zrotate_basis(nfs_ctx* c, int p, int q, int k, const std::vector<double>& z, bool with_mv) {
  const long long vstride = (long long)c->vcap * c->N;
  if (c->dY_len < z.size()) {
    if (c->dY) cudaFree(c->dY);
    c->dY = nullptr;
    c->dY_len = 0;
    TRY(dalloc(c, &c->dY, z.size()));
    c->dY_len = z.size();
  }
  CK(cudaMemcpyAsync(c->dY, z.data(), z.size() * sizeof(double), cudaMemcpyHostToDevice, c->work));
  CK(nfs::zrotate(c->V + p * vstride, q, c->dY, k, c->N, c->work));
  if (with_mv) CK(nfs::zrotate(c->MV + p * vstride, q, c->dY, k, c->N, c->work));
  CK(cudaStreamSynchronize(c->work));
  c->launches += with_mv ? 2 : 1;
  return NFS_OK;
}

// Largest loss of A_r-orthogonality removed with the FP32 shadow update; a
// larger one is removed in FP64 (the shadow update's rounding, ~6e-8 of the
// coefficients, would otherwise reappear above orth_tol).
constexpr double kShadowMaxLoss = 1e-6;

// Thick-restart invert Lanczos on (B_r, A_r) for every problem of the
// context, in lock-step, on the work stream.  omega: host P x nev; Y: device
// P x nev x N or null; infos: P entries or null.  Returns the worst status.
// The Lanczos basis size for nev wanted pairs, and the device memory that an
// eigensolve of that size uses (basis, its shadows, reduction scratch, the
// restart rotation matrix), allocated here once: an eigensolve within an
// earlier reservation allocates nothing.
int lanczos_size(nfs_ctx* c, int nev) {
  int m = c->opt.ncv > 0 ? c->opt.ncv : default_ncv(c, nev);
  return (int)std::min<long long>(m, c->N - 1);
}
int reserve_lanczos(nfs_ctx* c, int m) {
  TRY(ensure_basis(c, m));
  TRY(ensure_scratch(c, lanczos_scratch_len(c->P, c->vcap)));
  const size_t need = (size_t)c->P * m * m;  // rotate(): m x keep and k x nev, both <= m x m
  if (c->dY_len < need) {
    if (c->dY) cudaFree(c->dY);
    c->dY = nullptr;
    c->dY_len = 0;
    TRY(dalloc(c, &c->dY, need));
    c->dY_len = need;
  }
  return NFS_OK;
}

int eigs_core(nfs_ctx* c, int nev, double* omega, double2* Y, nfs_eigs_info* infos) {
  const int P = c->P;
  const long long N = c->N;
  const int m = lanczos_size(c, nev);
  if (m <= nev + 1) return NFS_EINVAL;
  TRY(reserve_lanczos(c, m));
  const long long vstride = (long long)c->vcap * N;
  cudaStream_t s = c->work;
  const long long mv32_0 = c->mv32, mv64_0 = c->mv64, launches_0 = c->launches;
  const double cg_0 = c->sec_cg, solve_0 = c->sec_solve, ritz_0 = c->sec_ritz, t_begin = now_s();
  const double recur_0 = c->sec_recur, orth_0 = c->sec_orth;
  const int nb = grid_blocks(P * N, 256);
  auto col = [&](double2* base, int p, int j) { return base + p * vstride + (long long)j * N; };

  // starting vectors, A_r-normalised (vector 0 of every basis)
  nfs::k_random_fill<<<nb, 256, 0, s>>>(c->V, N, vstride, P, c->opt.seed);
  CK(cudaGetLastError());
  c->launches += 1;
  for (int p = 0; p < P; ++p)
    CK(cudaMemcpyAsync(c->t64 + p * N, col(c->V, p, 0), N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  TRY(matvec<double>(c, s, c->t64, c->t64b));
  std::vector<double> nrm2;
  TRY(dots_re(c, s, c->t64, c->t64b, nrm2));
  std::vector<double> sc(P);
  for (int p = 0; p < P; ++p) {
    if (!(nrm2[p] > 0)) return NFS_EBREAKDOWN;
    sc[p] = 1.0 / std::sqrt(nrm2[p]);
  }
  TRY(put_small(c, s, P, sc));
  nfs::k_store_basis_vector<<<nb, 256, 0, s>>>(c->t64, c->t64b, c->d_small + P, c->V, c->MV, c->V32, c->MV32, c->MV32lo,
                                               vstride, 0, N, P, nullptr);
  CK(cudaGetLastError());
  c->launches += 1;

  const int check_every = 5;
  std::vector<std::vector<double>> H(P, std::vector<double>((size_t)m * m, 0.0));
  std::vector<double> beta_last(P, 0.0);
  std::vector<int> active(P, 1), jm(P, 0), nconv(P, 0), steps(P, 0), restarts_p(P, 0), reorths(P, 0);
  std::vector<int> full_reorths(P, 0);  // steps that needed the FP64 fallback
  std::vector<long long> cg_total(P, 0);
  std::vector<int> status(P, NFS_OK);
  int jstart = 0, local_lo = 0, restarts = 0;
  std::vector<double> theta, Z, coef, coef2, d, bb;
  double2* w = c->x64;    // new Krylov vectors (P x N)
  double2* Mw = c->t64b;  // A_r w
  int* d_active = c->d_flags;
  auto leading = [&](int p, int k) {
    std::vector<double> A((size_t)k * k);
    for (int r = 0; r < k; ++r)
      for (int q = 0; q < k; ++q) A[(size_t)r * k + q] = H[p][(size_t)r * m + q];
    return A;
  };
  auto any_active = [&]() {
    for (int p = 0; p < P; ++p)
      if (active[p]) return true;
    return false;
  };
  // One Lanczos run over the active problems from basis position jstart
  // until the nwant largest Ritz pairs of each have converged (thick restarts
  // when the basis fills).
  auto run = [&](int nwant) -> int {
  const int keep = std::min(m - 1, std::max(nwant + 1, nwant + (m - nwant) / 2));
  TRY(put_flags(c, s, 0, active));
  while (any_active()) {
    for (int j = jstart; j < m && any_active(); ++j) {
      // w = A_r^{-1} B_r v_j (CG); A_r w = B_r v_j
      TRY(apply_Br_basis(c, j, Mw));
      SolveOut so;
      CK(cudaStreamSynchronize(s));
      const double ts = now_s();
      TRY(solve(c, Mw, w, true, active, so));
      CK(cudaStreamSynchronize(s));
      c->sec_solve += now_s() - ts;
      // A_r w = B_r v_j - r with r the solve's final residual (the refined
      // FP64 residual in mixed contexts): the right-hand side alone would
      // carry the residual into A_r V, where the recurrence amplifies it like
      // the Lanczos polynomials; on long runs over degenerate spectra that
      // drift corrupted the orthogonality measure, the re-orthogonalisation
      // and the projected matrix
      TRY(sub64(c, s, Mw, c->r64, Mw));
      for (int p = 0; p < P; ++p) {
        if (!active[p]) continue;
        if (so.status[p] == NFS_EBREAKDOWN) {
          if (trace_lanczos())
            std::fprintf(stderr, "nfs lanczos: problem %d step %d (j %d): CG breakdown after %d iterations, "
                         "relres %.3e\n", p, steps[p] + 1, j, so.iters[p], so.relres[p]);
          return NFS_EBREAKDOWN;
        }
        cg_total[p] += so.iters[p];
        ++steps[p];
      }
      // FP64 three-term recurrence (after a restart: the arrow of kept Ritz
      // vectors) in the A_r inner product
      const int nl = j - local_lo + 1;
      const double tr0 = now_s();
      TRY(multi_dot(c, c->MV, local_lo, nl, w, coef, d_active));
      TRY(multi_axpy(c, w, Mw, local_lo, nl, coef, d_active));
      std::vector<double> alpha(P);
      for (int p = 0; p < P; ++p) {
        alpha[p] = coef[(size_t)p * 2 * nl + 2 * (j - local_lo)];
        if (!active[p]) continue;
        // the first step after a thick restart (or of a deflation check):
        // the couplings of the continuation vector to the kept (or locked)
        // vectors as measured, v_i^* B_r v_j, instead of their values in exact
        // arithmetic (beta times the last row of the Ritz vectors, or zero).
        // On long runs over degenerate spectra the two drift apart, and the
        // projected matrix must be the projection the orthogonalisation used
        // (else spurious Ritz values appear, even outside the spectrum).
        if (local_lo == 0 && j == jstart && j > 0)
          for (int i = 0; i < j; ++i)
            H[p][(size_t)i * m + j] = H[p][(size_t)j * m + i] = coef[(size_t)p * 2 * nl + 2 * i];
      }
      TRY(dots_re(c, s, w, Mw, bb));
      const std::vector<double> bb_recur = bb;
      std::vector<double> loss_first(P, 0.0);
      const double tr1 = now_s();
      c->sec_recur += tr1 - tr0;
      // Partial re-orthogonalisation: every step, measure the loss of
      // A_r-orthogonality against the older vectors [0, local_lo) with exact
      // inner products (double-single arithmetic on the split shadows); when
      // it exceeds orth_tol, remove those components (the vectors [local_lo,
      // j] were just orthogonalised in FP64 by the recurrence).  The update
      // is formed in FP32, exact enough while the coefficients are small
      // (loss <= kShadowMaxLoss); a larger loss is removed in FP64, and a
      // very large one (a coupling after a restart) takes a second pass.
      if (local_lo > 0) {
        std::vector<int> reorth(P, 0);
        for (int pass = 0; pass < 3; ++pass) {
          TRY(exact_dots(c, local_lo, w, d, d_active));
          bool any_re = false, big = false, big_loss = false;
          for (int p = 0; p < P; ++p) {
            reorth[p] = 0;
            if (!active[p]) continue;
            double loss = 0.0;
            for (int i = 0; i < local_lo; ++i)
              loss = std::max(loss, std::hypot(d[(size_t)p * 2 * local_lo + 2 * i], d[(size_t)p * 2 * local_lo + 2 * i + 1]));
            loss /= std::sqrt(std::max(bb[p], 1e-300));
            if (pass == 0) loss_first[p] = loss;
            reorth[p] = pass == 0 ? loss > c->opt.orth_tol : loss > 1e-3 * c->opt.orth_tol + 1e-13;
            any_re = any_re || reorth[p];
            big = big || (reorth[p] && loss > 1e-3);
            big_loss = big_loss || (reorth[p] && loss > kShadowMaxLoss);
            if (reorth[p] && pass == 0) ++reorths[p];
          }
          if (!any_re) break;
          TRY(put_flags(c, s, P, reorth));
          if (big_loss) {
            // a loss this large would come back from an FP32 update (its
            // rounding is ~6e-8 of the coefficients): remove the components
            // in FP64, with coefficients v_i^* A_r w from the stored A_r V
            TRY(multi_dot(c, c->MV, 0, local_lo, w, coef2, c->d_flags + P));
            TRY(multi_axpy(c, w, Mw, 0, local_lo, coef2, c->d_flags + P));
            for (int p = 0; p < P; ++p)
              if (reorth[p]) ++full_reorths[p];
          } else {
            nfs::k_shadow_axpy<<<dim3(grid_blocks(N, 256), P), 256, (size_t)local_lo * sizeof(float2), s>>>(
                w, Mw, c->V32, c->MV32, vstride, c->dscratch + off_fin(c), local_lo, N, c->d_flags + P);
            CK(cudaGetLastError());
            c->launches += 1;
          }
          TRY(dots_re(c, s, w, Mw, bb));
          if (!big) break;
        }
      }
      c->sec_orth += now_s() - tr1;
      if (trace_lanczos())
        for (int p = 0; p < P; ++p)
          if (active[p])
            std::fprintf(stderr, "nfs lanczos: problem %d step %d (j %d, lo %d): alpha %.17e beta2 %.6e -> %.6e "
                         "loss %.3e cg %d relres %.3e fp64-reorth %d\n", p, steps[p], j, local_lo, alpha[p],
                         bb_recur[p], bb[p], loss_first[p], so.iters[p], so.relres[p], full_reorths[p]);
      for (int p = 0; p < P; ++p) {
        if (!active[p]) continue;
        if (!(bb[p] > 0)) return NFS_EBREAKDOWN;
        const double beta = std::sqrt(bb[p]);
        H[p][(size_t)j * m + j] = alpha[p];
        if (j + 1 < m) H[p][(size_t)(j + 1) * m + j] = H[p][(size_t)j * m + j + 1] = beta;
        beta_last[p] = beta;
        sc[p] = 1.0 / beta;
      }
      TRY(put_small(c, s, P, sc));
      nfs::k_store_basis_vector<<<nb, 256, 0, s>>>(w, Mw, c->d_small + P, c->V, c->MV, c->V32, c->MV32,
                                                   c->MV32lo, vstride, j + 1, N, P, d_active);
      CK(cudaGetLastError());
      c->launches += 1;
      local_lo = j;
      // Ritz values of the leading (j+1) x (j+1) block; residual |beta z_last|
      const int k = j + 1;
      if (k >= nwant + 1 && ((k - jstart) % check_every == 0 || j == m - 1)) {
        bool changed = false;
        for (int p = 0; p < P; ++p) {
          if (!active[p]) continue;
          std::vector<double> zl;
          const double th0 = now_s();
          const bool ok = nfs::host::sym_eig(k, leading(p, k), theta, zl, true);
          c->sec_ritz += now_s() - th0;
          if (!ok) return NFS_EBREAKDOWN;
          int nc = 0;
          for (int i = 0; i < nwant; ++i) {
            const int cc = k - 1 - i;  // largest theta first
            if (std::fabs(beta_last[p] * zl[cc]) <= c->opt.eig_tol * std::fabs(theta[cc])) ++nc;
          }
          nconv[p] = std::min(nc, nev);
          if (nc == nwant) {
            jm[p] = k;
            active[p] = 0;
            changed = true;
          }
        }
        if (changed) TRY(put_flags(c, s, 0, active));
      }
    }
    if (!any_active()) break;
    if (restarts >= c->opt.max_restarts) {
      for (int p = 0; p < P; ++p)
        if (active[p]) {
          status[p] = NFS_ENOCONV;
          jm[p] = m;
          active[p] = 0;
        }
      break;
    }
    // thick restart of every unconverged problem: keep the `keep` largest
    // Ritz pairs of its full basis
    std::vector<double> Ycm((size_t)P * m * keep, 0.0);
    std::vector<std::vector<double>> th(P), zz(P);
    for (int p = 0; p < P; ++p) {
      if (!active[p]) continue;
      if (!nfs::host::sym_eig(m, leading(p, m), th[p], zz[p])) return NFS_EBREAKDOWN;
      for (int i = 0; i < keep; ++i)
        for (int r = 0; r < m; ++r) Ycm[(size_t)p * m * keep + (size_t)i * m + r] = zz[p][(size_t)r * m + (m - 1 - i)];
    }
    TRY(rotate(c, c->V, m, Ycm, keep, d_active));
    TRY(rotate(c, c->MV, m, Ycm, keep, d_active));
    for (int p = 0; p < P; ++p) {
      if (!active[p]) continue;
      CK(cudaMemcpyAsync(col(c->V, p, keep), col(c->V, p, m), N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(col(c->MV, p, keep), col(c->MV, p, m), N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
      std::fill(H[p].begin(), H[p].end(), 0.0);
      for (int i = 0; i < keep; ++i) {
        H[p][(size_t)i * m + i] = th[p][m - 1 - i];
        const double sres = beta_last[p] * zz[p][(size_t)(m - 1) * m + (m - 1 - i)];
        H[p][(size_t)keep * m + i] = H[p][(size_t)i * m + keep] = sres;
      }
      ++restarts_p[p];
    }
    TRY(refresh_shadows(c, 0, keep + 1));
    jstart = keep;
    local_lo = 0;
    ++restarts;
  }
  return NFS_OK;
  };
  TRY(run(nev));

  // Deflation checks.  A single start vector has one component in each
  // eigenspace, so the Krylov space holds one vector of a degenerate
  // eigenvalue; its other copies enter only through rounding, possibly after
  // the wanted pairs have converged.  Each check locks the nev converged Ritz
  // vectors (basis positions 0..nev-1, decoupled: H = diag(theta)), restarts
  // from a random vector A_r-orthogonal to them and runs until the next
  // eigenvalue, the largest of the operator on their A_r-orthogonal
  // complement, has converged too.  If it belongs among the nev largest (a
  // missed copy), another check follows.
  std::vector<int> one(P, 0), verified(P, 0), dchecks(P, 0);
  for (int round = 0; round < c->opt.deflation_checks; ++round) {
    std::vector<int> part(P, 0);
    bool anyp = false;
    for (int p = 0; p < P; ++p) {
      part[p] = status[p] == NFS_OK && !verified[p];
      anyp = anyp || part[p];
    }
    if (!anyp) break;
    for (int p = 0; p < P; ++p) {
      if (!part[p]) continue;
      const int k = jm[p];
      if (!nfs::host::sym_eig(k, leading(p, k), theta, Z)) return NFS_EBREAKDOWN;
      std::vector<double> Ycm((size_t)P * k * nev, 0.0);
      for (int i = 0; i < nev; ++i)
        for (int r = 0; r < k; ++r) Ycm[(size_t)p * k * nev + (size_t)i * k + r] = Z[(size_t)r * k + (k - 1 - i)];
      std::fill(one.begin(), one.end(), 0);
      one[p] = 1;
      TRY(put_flags(c, s, P, one));
      TRY(rotate(c, c->V, k, Ycm, nev, c->d_flags + P));
      TRY(rotate(c, c->MV, k, Ycm, nev, c->d_flags + P));
      std::fill(H[p].begin(), H[p].end(), 0.0);
      for (int i = 0; i < nev; ++i) H[p][(size_t)i * m + i] = theta[k - 1 - i];
      beta_last[p] = 0.0;
      ++dchecks[p];
    }
    active = part;
    TRY(put_flags(c, s, 0, active));
    TRY(refresh_shadows(c, 0, nev));
    // the new start vector, A_r-orthogonalised twice against the locked ones
    nfs::k_random_fill<<<nb, 256, 0, s>>>(c->V + (long long)nev * N, N, vstride, P,
                                          c->opt.seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(round + 1));
    CK(cudaGetLastError());
    c->launches += 1;
    for (int p = 0; p < P; ++p)
      CK(cudaMemcpyAsync(w + p * N, col(c->V, p, nev), N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    TRY(matvec<double>(c, s, w, Mw));
    for (int pass = 0; pass < 2; ++pass) {
      TRY(multi_dot(c, c->MV, 0, nev, w, coef, d_active));
      TRY(multi_axpy(c, w, Mw, 0, nev, coef, d_active));
    }
    TRY(dots_re(c, s, w, Mw, bb));
    for (int p = 0; p < P; ++p) {
      if (active[p] && !(bb[p] > 0)) return NFS_EBREAKDOWN;
      sc[p] = active[p] ? 1.0 / std::sqrt(bb[p]) : 0.0;
    }
    TRY(put_small(c, s, P, sc));
    nfs::k_store_basis_vector<<<nb, 256, 0, s>>>(w, Mw, c->d_small + P, c->V, c->MV, c->V32, c->MV32, c->MV32lo,
                                                 vstride, nev, N, P, d_active);
    CK(cudaGetLastError());
    c->launches += 1;
    jstart = nev;
    local_lo = 0;
    TRY(run(nev + 1));
    // a locked set is confirmed when the new block adds nothing to the nev
    // largest Ritz pairs (its share of their invariant subspace is ~0)
    for (int p = 0; p < P; ++p) {
      if (!part[p] || status[p] != NFS_OK) continue;
      const int k = jm[p];
      if (!nfs::host::sym_eig(k, leading(p, k), theta, Z)) return NFS_EBREAKDOWN;
      double mass = 0.0;
      for (int i = 0; i < nev; ++i)
        for (int r = nev; r < k; ++r) mass += Z[(size_t)r * k + (k - 1 - i)] * Z[(size_t)r * k + (k - 1 - i)];
      verified[p] = mass < 0.5;
    }
  }

  // results from each problem's leading jm x jm block: omega ascending = theta descending
  const double tv0 = now_s();
  int worst = NFS_OK;
  for (int p = 0; p < P; ++p) {
    const int k = jm[p];
    if (!nfs::host::sym_eig(k, leading(p, k), theta, Z)) return NFS_EBREAKDOWN;
    double maxres = 0.0;
    for (int i = 0; i < nev; ++i) {
      const int cc = k - 1 - i;
      omega[(size_t)p * nev + i] = 1.0 / theta[cc];
      maxres = std::max(maxres, std::fabs(beta_last[p] * Z[(size_t)(k - 1) * k + cc]) / std::fabs(theta[cc]));
    }
    if (status[p] == NFS_OK) {
      // a Rayleigh-Ritz on the span of the nev Ritz vectors with the true
      // inner products: second-order accurate eigenvalues for copies found by
      // deflation checks, and values that stay inside the spectrum even where
      // the basis has lost A_r-orthogonality
      std::vector<double> Ycm((size_t)P * k * nev, 0.0);
      for (int i = 0; i < nev; ++i)
        for (int r = 0; r < k; ++r) Ycm[(size_t)p * k * nev + (size_t)i * k + r] = Z[(size_t)r * k + (k - 1 - i)];
      std::fill(one.begin(), one.end(), 0);
      one[p] = 1;
      TRY(put_flags(c, s, P, one));
      TRY(rotate(c, c->V, k, Ycm, nev, c->d_flags + P));
      std::vector<double> th2, zc;
      TRY(final_rayleigh_ritz(c, p, nev, c->d_flags + P, th2, zc));
      for (int i = 0; i < nev; ++i) omega[(size_t)p * nev + i] = 1.0 / th2[i];
      TRY(zrotate_basis(c, p, nev, nev, zc, false));
      if (Y) {
        CK(cudaMemcpyAsync(Y + (long long)p * nev * N, col(c->V, p, 0), (size_t)nev * N * sizeof(double2),
                           cudaMemcpyDeviceToDevice, s));
        CK(cudaStreamSynchronize(s));
      }
    } else if (Y) {
      // Ritz vectors of problem p: rotate its basis (only p flagged), then copy
      std::vector<double> Ycm((size_t)P * k * nev, 0.0);
      for (int i = 0; i < nev; ++i)
        for (int r = 0; r < k; ++r) Ycm[(size_t)p * k * nev + (size_t)i * k + r] = Z[(size_t)r * k + (k - 1 - i)];
      std::fill(one.begin(), one.end(), 0);
      one[p] = 1;
      TRY(put_flags(c, s, P, one));
      TRY(rotate(c, c->V, k, Ycm, nev, c->d_flags + P));
      CK(cudaMemcpyAsync(Y + (long long)p * nev * N, col(c->V, p, 0), (size_t)nev * N * sizeof(double2),
                         cudaMemcpyDeviceToDevice, s));
    }
    if (infos) {
      nfs_eigs_info& in = infos[p];
      in.lanczos_steps = steps[p];
      in.restarts = restarts_p[p];
      in.cg_iterations = cg_total[p];
      in.matvecs_c64 = (c->mv32 - mv32_0) / P;
      in.matvecs_c128 = (c->mv64 - mv64_0) / P;
      in.nconv = status[p] == NFS_OK ? nev : nconv[p];
      in.max_ritz_residual = maxres;
      in.status = status[p];
      in.kernel_launches = c->launches - launches_0;
      in.seconds_total = now_s() - t_begin;
      in.seconds_cg = c->sec_cg - cg_0;
      in.seconds_refine = (c->sec_solve - solve_0) - (c->sec_cg - cg_0);
      in.seconds_ritz = c->sec_ritz - ritz_0;
      in.seconds_recurrence = c->sec_recur - recur_0;
      in.seconds_orth = c->sec_orth - orth_0;
      in.seconds_vectors = now_s() - tv0;
      in.reorthogonalisations = reorths[p];
      in.deflation_checks = dchecks[p];
    }
    if (status[p] != NFS_OK) worst = status[p];
  }
  CK(cudaStreamSynchronize(s));
  return worst;
}

// Order the context's work stream after everything already queued on the
// caller's stream.
int join_caller(nfs_ctx* c) {
  CK(cudaEventRecord(c->ev, c->stream));
  CK(cudaStreamWaitEvent(c->work, c->ev, 0));
  return NFS_OK;
}

void free_ctx(nfs_ctx* c) {
  if (!c) return;
  for (GraphEntry& g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (GmresGraph& g : c->gm_graphs) cudaGraphExecDestroy(g.exec);
  void* ptrs[] = {c->lam64, c->lam32, c->tw64[0], c->tw64[1], c->tw64[2], c->tw32[0], c->tw32[1], c->tw32[2],
                  c->mat64, c->mat32, c->basis64, c->bloch64, c->lamdf, c->twdf[0], c->twdf[1], c->twdf[2], c->matdf,
                  c->basisdf, c->fld, c->x64, c->r64, c->p64, c->Ap64, c->t64, c->t64b, c->x32, c->r32,
                  c->p32, c->p32b, c->Ap32, c->st, c->d_small, c->d_flags, c->dscratch, c->V, c->MV, c->V32, c->MV32,
                  c->MV32lo, c->dY, c->binv64, c->zv, c->gv, c->zY};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->h_small) cudaFreeHost(c->h_small);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->hscratch) cudaFreeHost(c->hscratch);
  if (c->work) cudaStreamDestroy(c->work);
  if (c->ev) cudaEventDestroy(c->ev);
  delete c;
}

// --- set-up -------------------------------------------------------------------

struct Prepared {
  double kd[3];
  std::vector<double2> lam;
  std::vector<double> m64;
};

int check_options(const nfs_options& o) {
  if (o.precision != NFS_PREC_FP64 && o.precision != NFS_PREC_MIXED) return NFS_EINVAL;
  if (!(o.cg_tol > 0) || o.cg_maxit <= 0 || !(o.eig_tol > 0) || o.max_restarts < 0) return NFS_EINVAL;
  if (!(o.orth_tol >= 0) || !(o.orth_tol < 1)) return NFS_EINVAL;
  if (o.deflation_checks < 0 || o.deflation_checks > 16) return NFS_EINVAL;
  if (o.precision == NFS_PREC_MIXED && (!(o.inner_tol > 0) || o.inner_tol >= 1 || o.max_refine <= 0))
    return NFS_EINVAL;
  if (!(o.alpha != 0.0) || !(o.beta != 0.0)) return NFS_EBASIS;
  return NFS_OK;
}

// Validate one problem and build its tables and material (host, FP64): the
// Lemma (lem:nonsingular_full_rank) and the Assumption (eq. assump).
int prepare_problem(const int grid[3], const double* lattice, const double k[3], const nfs_material* mat,
                    const nfs_options& o, Prepared& out, double delta[3]) {
  if (!grid || !k || !mat || !mat->eps || !mat->gamma) return NFS_EINVAL;
  for (int l = 0; l < 3; ++l)
    if (grid[l] <= 0) return NFS_EINVAL;
  if (mat->kind != NFS_MEDIUM_CHIRAL && mat->kind != NFS_MEDIUM_PSEUDOCHIRAL) return NFS_EINVAL;
  if (mat->kind == NFS_MEDIUM_PSEUDOCHIRAL &&
      (mat->axis_a < 0 || mat->axis_a > 2 || mat->axis_b < 0 || mat->axis_b > 2 || mat->axis_a == mat->axis_b))
    return NFS_EINVAL;
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
  const int nn[3] = {n1, n2, n3};
  bool all_int = true;
  for (int l = 0; l < 3; ++l) {
    if (!std::isfinite(k[l])) return NFS_EINVAL;
    out.kd[l] = k[l] * a_len[l];
    delta[l] = a_len[l] / nn[l];
    if (std::fabs(out.kd[l] - std::round(out.kd[l])) > 1e-12) all_int = false;
  }
  if (all_int) return NFS_EKPOINT;

  // Lambda tables (thm:SchurDecomp_Ci): (exp(i 2 pi (i + k.a)/m) - 1) / delta,
  // real part written as -2 sin^2(theta/2) to avoid cancellation.
  out.lam.assign(n1 + n2 + n3, make_double2(0, 0));
  {
    int off = 0;
    for (int l = 0; l < 3; ++l) {
      for (int i = 0; i < nn[l]; ++i) {
        const double th = 2.0 * M_PI * (i + out.kd[l]) / nn[l];
        const double sh = std::sin(0.5 * th);
        out.lam[off + i] = make_double2(-2.0 * sh * sh / delta[l], std::sin(th) / delta[l]);
      }
      off += nn[l];
    }
  }
  // Lemma: Lambda_q > 0 and Lambda_p != 0 at every voxel
  {
    const double al = o.alpha, be = o.beta;
    double minq = INFINITY, minp = INFINITY;
    for (int i3 = 0; i3 < n3; ++i3)
      for (int i2 = 0; i2 < n2; ++i2)
        for (int i1 = 0; i1 < n1; ++i1) {
          const double2 a1 = out.lam[i1], a2 = out.lam[n1 + i2], a3 = out.lam[n1 + n2 + i3];
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
  out.m64.assign(mat_len, 0.0);
  double* inv_phi = out.m64.data();
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
  return NFS_OK;
}

// Host-side validation and tables for P problems that share grid, medium
// kind, axis pair and mu-ness (no CUDA call).
int prepare_class(int P, const int grid[3], const double* const* lattices, const double* const* ks,
                  const nfs_material* const* mats, const nfs_options& o, std::vector<Prepared>& prep,
                  double delta[3]) {
  prep.assign(P, Prepared{});
  for (int p = 0; p < P; ++p) TRY(prepare_problem(grid, lattices[p], ks[p], mats[p], o, prep[p], delta));
  const nfs_material* m0 = mats[0];
  for (int p = 1; p < P; ++p) {
    if (mats[p]->kind != m0->kind || (mats[p]->mu != nullptr) != (m0->mu != nullptr)) return NFS_EINVAL;
    if (m0->kind == NFS_MEDIUM_PSEUDOCHIRAL && (mats[p]->axis_a != m0->axis_a || mats[p]->axis_b != m0->axis_b))
      return NFS_EINVAL;
  }
  return NFS_OK;
}

// The device side of a context for a prepared class.
int setup_class(nfs_ctx** out, int P, const int grid[3], const nfs_material* const* mats,
                const std::vector<Prepared>& prep, const double delta[3], const nfs_options& o) {
  *out = nullptr;
  const nfs_material* m0 = mats[0];
  int dev = 0;
  CK(cudaGetDevice(&dev));
  nfs_ctx* c = new (std::nothrow) nfs_ctx();
  if (!c) return NFS_ENOMEM;
  const int n1 = grid[0], n2 = grid[1], n3 = grid[2];
  c->n1 = n1; c->n2 = n2; c->n3 = n3; c->nl = n1 + n2 + n3;
  c->n = (long long)n1 * n2 * n3;
  c->N = 4 * c->n;
  c->P = P;
  for (int l = 0; l < 3; ++l) c->delta[l] = delta[l];
  c->opt = o;
  c->stream = (cudaStream_t)o.stream;
  c->kind = m0->kind;
  c->ax_a = c->kind == NFS_MEDIUM_CHIRAL ? 0 : m0->axis_a;
  c->ax_b = c->kind == NFS_MEDIUM_CHIRAL ? 1 : m0->axis_b;
  c->has_mu = m0->mu != nullptr;
  c->gam_len = (c->kind == NFS_MEDIUM_CHIRAL) ? 3 * c->n : c->n;
  c->mat_len = (long long)prep[0].m64.size();

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

  CKC(cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking));
  CKC(cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming));
  const int nl = c->nl;
  {
    std::vector<double2> lam((size_t)P * nl);
    std::vector<float2> lam32((size_t)P * nl);
    for (int p = 0; p < P; ++p)
      for (int i = 0; i < nl; ++i) {
        lam[(size_t)p * nl + i] = prep[p].lam[i];
        lam32[(size_t)p * nl + i] = make_float2((float)prep[p].lam[i].x, (float)prep[p].lam[i].y);
      }
    TRYC(dalloc(c, &c->lam64, (size_t)P * nl));
    TRYC(dalloc(c, &c->lam32, (size_t)P * nl));
    CKC(cudaMemcpy(c->lam64, lam.data(), lam.size() * sizeof(double2), cudaMemcpyHostToDevice));
    CKC(cudaMemcpy(c->lam32, lam32.data(), lam32.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  const int nn[3] = {n1, n2, n3};
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
  {
    const size_t ml = (size_t)c->mat_len;
    TRYC(dalloc(c, &c->mat64, (size_t)P * ml));
    TRYC(dalloc(c, &c->mat32, (size_t)P * ml));
    std::vector<float> m32(ml);
    for (int p = 0; p < P; ++p) {
      for (size_t i = 0; i < ml; ++i) m32[i] = (float)prep[p].m64[i];
      CKC(cudaMemcpy(c->mat64 + (size_t)p * ml, prep[p].m64.data(), ml * sizeof(double), cudaMemcpyHostToDevice));
      CKC(cudaMemcpy(c->mat32 + (size_t)p * ml, m32.data(), ml * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  {
    std::vector<double2> d((size_t)P * nl);
    c->kd.assign((size_t)3 * P, 0.0);
    for (int p = 0; p < P; ++p)
      for (int l = 0, off = 0; l < 3; off += nn[l], ++l) {
        c->kd[3 * p + l] = prep[p].kd[l];
        for (int j = 0; j < nn[l]; ++j) {
          const double th = 2.0 * M_PI * prep[p].kd[l] * j / nn[l];
          d[(size_t)p * nl + off + j] = make_double2(std::cos(th), std::sin(th));
        }
      }
    TRYC(dalloc(c, &c->bloch64, (size_t)P * nl));
    CKC(cudaMemcpy(c->bloch64, d.data(), d.size() * sizeof(double2), cudaMemcpyHostToDevice));
  }
  TRYC(dalloc(c, &c->basis64, (size_t)P * 6 * c->n));
  CKC(nfs::basis_table_launch(c->lam64, n1, n2, n3, o.alpha, o.beta, c->basis64, P, nl, 6 * c->n, 0));
  if (o.precision == NFS_PREC_MIXED) {
    TRYC(dalloc(c, &c->lamdf, (size_t)P * nl));
    CKC(nfs::double_to_df(reinterpret_cast<const double*>(c->lam64), reinterpret_cast<nfs::df*>(c->lamdf),
                          2LL * P * nl, 0));
    for (int l = 0; l < 3; ++l) {
      TRYC(dalloc(c, &c->twdf[l], nn[l]));
      CKC(nfs::double_to_df(reinterpret_cast<const double*>(c->tw64[l]), reinterpret_cast<nfs::df*>(c->twdf[l]),
                            2LL * nn[l], 0));
    }
    TRYC(dalloc(c, &c->matdf, (size_t)P * c->mat_len));
    CKC(nfs::double_to_df(c->mat64, c->matdf, (long long)P * c->mat_len, 0));
    TRYC(dalloc(c, &c->basisdf, (size_t)P * 6 * c->n));
    CKC(nfs::double_to_df(reinterpret_cast<const double*>(c->basis64), reinterpret_cast<nfs::df*>(c->basisdf),
                          2LL * P * 6 * c->n, 0));
  }
  const size_t PN = (size_t)P * c->N;
  TRYC(dalloc(c, (double2**)&c->fld, (size_t)P * 6 * c->n));
  TRYC(dalloc(c, &c->x64, PN));
  TRYC(dalloc(c, &c->r64, PN));
  TRYC(dalloc(c, &c->p64, PN));
  TRYC(dalloc(c, &c->Ap64, PN));
  TRYC(dalloc(c, &c->t64, PN));
  TRYC(dalloc(c, &c->t64b, PN));
  if (o.precision == NFS_PREC_MIXED) {
    TRYC(dalloc(c, &c->x32, PN));
    TRYC(dalloc(c, &c->r32, PN));
    TRYC(dalloc(c, &c->p32, PN));
    TRYC(dalloc(c, &c->Ap32, PN));
    if (nfs::cg_needs_p_out<float>(n1)) TRYC(dalloc(c, &c->p32b, PN));
  }
  TRYC(dalloc(c, &c->st, P));
  CKC(cudaMallocHost((void**)&c->st_host, (size_t)P * sizeof(CGState)));
  std::memset(c->st_host, 0, (size_t)P * sizeof(CGState));
  CKC(cudaMemset(c->st, 0, (size_t)P * sizeof(CGState)));
  TRYC(dalloc(c, &c->d_small, (size_t)kSmallSlots * P));
  CKC(cudaMallocHost((void**)&c->h_small, (size_t)kSmallSlots * P * sizeof(double)));
  TRYC(dalloc(c, &c->d_flags, (size_t)kFlagSlots * P));
  CKC(cudaMallocHost((void**)&c->h_flags, (size_t)kFlagSlots * P * sizeof(int)));
  TRYC(ensure_scratch(c, (size_t)kRedBlocks * 2 * 64 * P + 4096));
  CKC(nfs::matvec_prepare<double>(n1, n2, n3));
  CKC(nfs::matvec_prepare<float>(n1, n2, n3));
  if (o.precision == NFS_PREC_MIXED) CKC(nfs::matvec_prepare<nfs::df>(n1, n2, n3));
  CKC(nfs::grad_prepare(n1, n2, n3));
  CKC(nfs::fields_prepare(n1, n2, n3));
  // an explicit basis size: the eigensolver's memory is taken here, so that
  // no later call allocates
  if (o.ncv > 0) TRYC(reserve_lanczos(c, (int)std::min<long long>(o.ncv, c->N - 1)));
  CKC(cudaDeviceSynchronize());
#undef TRYC
#undef CKC
  *out = c;
  return NFS_OK;
}

nfs_options resolved_options(const nfs_options* opt) {
  nfs_options o;
  nfs_default_options(&o);
  if (opt) o = *opt;
  return o;
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
  o->inner_tol = 1e-6;
  o->max_refine = 8;
  o->eig_tol = 1e-10;
  o->ncv = 0;
  o->max_restarts = 200;
  o->orth_tol = 1e-10;
  o->deflation_checks = 0;
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
  if (!grid || !k || !mat) return NFS_EINVAL;
  const nfs_options o = resolved_options(opt);
  TRY(check_options(o));
  const double* lat[1] = {lattice};
  const double* ks[1] = {k};
  const nfs_material* ms[1] = {mat};
  std::vector<Prepared> prep;
  double delta[3] = {0, 0, 0};
  TRY(prepare_class(1, grid, lat, ks, ms, o, prep, delta));
  return setup_class(out, 1, grid, ms, prep, delta, o);
}

extern "C" void nfs_destroy(nfs_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  cudaStreamSynchronize(c->work);
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
  if (c->binv64) return NFS_EUNSUPPORTED;  // no A_r outside the Assumption
  if (((uintptr_t)u | (uintptr_t)Au) & 15) return NFS_EINVAL;  // 16-byte vector access
  if (dtype == NFS_C128) return matvec<double>(c, c->stream, (const double2*)u, (double2*)Au);
  if (dtype == NFS_C64) return matvec<float>(c, c->stream, (const float2*)u, (float2*)Au);
  if (dtype == NFS_C128_DS) {
    if (!c->lamdf) return NFS_EINVAL;  // FP64 contexts hold no double-single tables
    return matvec_refine(c, c->stream, (const double2*)u, (double2*)Au, nullptr, 0);
  }
  return NFS_EINVAL;
}

extern "C" int nfs_matvec_passes(nfs_ctx* c, int dtype, int mask, const void* u, void* Au) {
  if (!c || mask <= 0 || mask > 7) return NFS_EINVAL;
  if (c->binv64) return NFS_EUNSUPPORTED;
  if ((mask & 1) && !u) return NFS_EINVAL;
  if ((mask & 4) && !Au) return NFS_EINVAL;
  if (((uintptr_t)u | (uintptr_t)Au) & 15) return NFS_EINVAL;
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
  if (c->binv64) return NFS_EUNSUPPORTED;
  nfs::k_apply_Br<<<grid_blocks(c->n * c->P, 256), 256, 0, c->stream>>>((const double2*)v, (double2*)out, c->lam64,
                                                                          c->n1, c->n2, c->n3, c->P);
  CK(cudaGetLastError());
  return NFS_OK;
}

extern "C" int nfs_cg_solve(nfs_ctx* c, const void* b, void* x, nfs_solve_info* info) {
  if (!c || !b || !x || b == x) return NFS_EINVAL;
  if (c->binv64) return NFS_EUNSUPPORTED;
  if (((uintptr_t)b | (uintptr_t)x) & 15) return NFS_EINVAL;
  TRY(join_caller(c));
  // the solve runs on the context's buffers (so that its CUDA graph is reused)
  const size_t bytes = (size_t)c->P * c->N * sizeof(double2);
  CK(cudaMemcpyAsync(c->t64b, b, bytes, cudaMemcpyDeviceToDevice, c->work));
  CK(cudaMemcpyAsync(c->t64, x, bytes, cudaMemcpyDeviceToDevice, c->work));
  SolveOut so;
  std::vector<int> active(c->P, 1);
  TRY(solve(c, c->t64b, c->t64, false, active, so));
  CK(cudaMemcpyAsync(x, c->t64, bytes, cudaMemcpyDeviceToDevice, c->work));
  CK(cudaStreamSynchronize(c->work));
  if (info) {
    info->iterations = so.iters[0];
    info->refinements = so.refines[0];
    info->rel_residual = so.relres[0];
    info->status = so.status[0];
  }
  return so.status[0];
}

extern "C" int nfs_residuals(nfs_ctx* c, int m, const double* omega, const void* Yv, double* res) {
  if (!c || m <= 0 || !omega || !Yv || !res) return NFS_EINVAL;
  if (c->binv64) return NFS_EUNSUPPORTED;
  if (c->P != 1) return NFS_EUNSUPPORTED;
  if ((uintptr_t)Yv & 15) return NFS_EINVAL;
  TRY(join_caller(c));
  cudaStream_t s = c->work;
  const long long n = c->n, N = c->N;
  const double2* Y = (const double2*)Yv;
  for (int j = 0; j < m; ++j) {
    const double2* y = Y + (long long)j * N;
    // A_r y (complex128 product) and B_r y, then |A_r y - omega B_r y| / |y|
    TRY(matvec<double>(c, s, y, c->t64b));
    nfs::k_apply_Br<<<grid_blocks(n, 256), 256, 0, s>>>(y, c->t64, c->lam64, c->n1, c->n2, c->n3, 1);
    nfs::k_residual_parts<<<kRedBlocks, kRedThreads, 0, s>>>(c->t64b, c->t64, y, omega[j], N, c->dscratch);
    CK(cudaGetLastError());
    c->launches += 2;
    CK(cudaMemcpyAsync(c->hscratch, c->dscratch, (size_t)2 * kRedBlocks * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double rr = 0.0, yy = 0.0;
    for (int b = 0; b < kRedBlocks; ++b) {
      rr += c->hscratch[2 * b];
      yy += c->hscratch[2 * b + 1];
    }
    if (!(yy > 0.0)) return NFS_EINVAL;
    res[j] = std::sqrt(rr / yy);
  }
  return NFS_OK;
}

namespace {
int nfsep_reserve(nfs_ctx* c, int nev);
}  // namespace

extern "C" int nfs_reserve(nfs_ctx* c, int nev) {
  if (!c || nev <= 0 || nev >= c->N / 2) return NFS_EINVAL;
  if (c->binv64) {
    TRY(nfsep_reserve(c, nev));
    CK(cudaDeviceSynchronize());
    return NFS_OK;
  }
  const int m = lanczos_size(c, nev);
  if (m <= nev + 1) return NFS_EINVAL;
  TRY(reserve_lanczos(c, m));
  CK(cudaDeviceSynchronize());
  return NFS_OK;
}

extern "C" int nfs_eigs(nfs_ctx* c, int nev, double* omega, void* Y, nfs_eigs_info* info) {
  if (!c || !omega || nev <= 0 || nev >= c->N / 2) return NFS_EINVAL;
  if (c->binv64) return NFS_EUNSUPPORTED;
  TRY(join_caller(c));
  return eigs_core(c, nev, omega, (double2*)Y, info);
}

extern "C" int nfs_eig_grad(nfs_ctx* c, int m, const double* weights, const void* Yv, double* d_eps,
                            double* d_gamma) {
  if (!c || m <= 0 || !weights || !Yv) return NFS_EINVAL;
  if (c->has_mu || c->P != 1 || c->binv64) return NFS_EUNSUPPORTED;
  TRY(join_caller(c));
  cudaStream_t s = c->work;
  const long long n = c->n, N = c->N;
  if (d_eps) CK(cudaMemsetAsync(d_eps, 0, 3 * n * sizeof(double), s));
  if (d_gamma) CK(cudaMemsetAsync(d_gamma, 0, c->gam_len * sizeof(double), s));
  const double2* Y = (const double2*)Yv;
  std::vector<double> yBy;
  for (int j = 0; j < m; ++j) {
    const double2* y = Y + (long long)j * N;
    nfs::k_apply_Br<<<grid_blocks(n, 256), 256, 0, s>>>(y, c->t64, c->lam64, c->n1, c->n2, c->n3, 1);
    CK(cudaGetLastError());
    TRY(dots_re(c, s, y, c->t64, yBy));
    if (!(yBy[0] != 0.0)) return NFS_EINVAL;
    const double scale = weights[j] / ((double)n * yBy[0]);
    nfs::MatvecArgs<double> a = margs<double>(c, y, nullptr, nullptr);
    a.stream = s;
    cudaError_t e = nfs::pass1_launch<double>(a);
    if (e != cudaSuccess) return cuda_fail(e, "grad pass 1");
    nfs::GradArgs g{};
    g.fld = (const double2*)c->fld; g.tw3 = c->tw64[2];
    g.inv_phi = c->mat64; g.gam = c->mat64 + 3 * n;
    g.kind = c->kind; g.ax_a = c->ax_a; g.ax_b = c->ax_b;
    g.n1 = c->n1; g.n2 = c->n2; g.n3 = c->n3;
    g.scale = scale; g.d_eps = d_eps; g.d_gamma = d_gamma; g.stream = s;
    e = nfs::grad_launch(g);
    if (e != cudaSuccess) return cuda_fail(e, "grad launch");
    c->launches += 2 + nfs::plane_pass_kernels<double>(c->n1);  // B_r, pass 1, gradient
  }
  CK(cudaStreamSynchronize(s));
  return NFS_OK;
}

extern "C" int nfs_eig_fields(nfs_ctx* c, int m, const void* Yv, void* Xv) {
  if (!c || m <= 0 || !Yv || !Xv) return NFS_EINVAL;
  if ((((uintptr_t)Yv) | ((uintptr_t)Xv)) & 15) return NFS_EINVAL;
  if (c->P != 1 || c->binv64) return NFS_EUNSUPPORTED;
  const long long n = c->n, N = c->N;
  const double2* Y = (const double2*)Yv;
  double2* X = (double2*)Xv;
  for (int j = 0; j < m; ++j) {
    // pass 1 of the complex128 product: the sqrt(n)-scaled untwisted (p, q),
    // transformed along x and y
    nfs::MatvecArgs<double> a = margs<double>(c, Y + (long long)j * N, nullptr, nullptr);
    cudaError_t e = nfs::pass1_launch<double>(a);
    if (e != cudaSuccess) return cuda_fail(e, "fields pass 1");
    nfs::FieldsArgs f{};
    f.fld = (const double2*)c->fld; f.tw3 = c->tw64[2]; f.bloch = c->bloch64;
    f.inv_phi = a.inv_phi; f.gam = a.gam; f.inv_mu = a.inv_mu;
    f.kind = c->kind; f.ax_a = c->ax_a; f.ax_b = c->ax_b;
    f.n1 = c->n1; f.n2 = c->n2; f.n3 = c->n3;
    f.X = X + (long long)j * 6 * n; f.stream = c->stream;
    e = nfs::fields_launch(f);
    if (e != cudaSuccess) return cuda_fail(e, "fields launch");
    c->launches += 1 + nfs::plane_pass_kernels<double>(c->n1);
  }
  return NFS_OK;
}

extern "C" int nfs_gep_residual(nfs_ctx* c, int m, const double* omega, const void* Xv, double* res) {
  if (!c || m <= 0 || !omega || !Xv || !res) return NFS_EINVAL;
  if (c->P != 1 || c->binv64) return NFS_EUNSUPPORTED;
  for (int j = 0; j < m; ++j)
    if (!(std::isfinite(omega[j]) && omega[j] != 0.0)) return NFS_EINVAL;
  const long long n = c->n;
  nfs::GepResidualArgs g{};
  g.inv_phi = c->mat64; g.gam = c->mat64 + 3 * n;
  g.inv_mu = c->has_mu ? c->mat64 + 3 * n + c->gam_len : nullptr;
  g.kind = c->kind; g.ax_a = c->ax_a; g.ax_b = c->ax_b;
  g.n1 = c->n1; g.n2 = c->n2; g.n3 = c->n3;
  for (int l = 0; l < 3; ++l) {
    g.inv_delta[l] = 1.0 / c->delta[l];
    const double th = 2.0 * M_PI * c->kd[l];
    g.wrap[l] = make_double2(std::cos(th), std::sin(th));
  }
  g.part = c->dscratch;
  const int blocks = (int)std::min<long long>(kRedBlocks, (n + 255) / 256);
  for (int j = 0; j < m; ++j) {
    g.X = (const double2*)Xv + (long long)j * 6 * n;
    g.omega = omega[j];
    cudaError_t e = nfs::gep_residual_launch(g, blocks, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "GEP residual launch");
    c->launches += 1;
    CK(cudaMemcpyAsync(c->hscratch, c->dscratch, (size_t)2 * blocks * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double r2 = 0.0, b2 = 0.0;
    for (int i = 0; i < blocks; ++i) {
      r2 += c->hscratch[2 * i];
      b2 += c->hscratch[2 * i + 1];
    }
    res[j] = std::sqrt(r2) / (std::fabs(omega[j]) * std::sqrt(b2));
  }
  return NFS_OK;
}

// --- media outside the Assumption: the NFSEP --------------------------------

namespace {

// M y (- sigma v) on the given stream: Sigma^{1/2}, pass 1, the B^{-1} z-pass,
// pass 3, halves exchanged and Sigma^{1/2} (t64 and Ap64 are its temporaries)
int nfsep_apply(nfs_ctx* c, cudaStream_t s, const double2* y, double2* out, const double2* v, double2 sigma) {
  cudaError_t e = nfs::nfsep_prescale(y, c->t64, c->lam64, c->n1, c->n2, c->n3, s);
  if (e != cudaSuccess) return cuda_fail(e, "nfsep prescale");
  nfs::MatvecArgs<double> a = margs<double>(c, c->t64, c->Ap64, nullptr);
  a.stream = s;
  e = nfs::pass1_launch<double>(a);
  if (e != cudaSuccess) return cuda_fail(e, "nfsep pass 1");
  e = nfs::nfsep_pass2((double2*)c->fld, c->binv64, c->tw64[2], c->n1, c->n2, c->n3, s);
  if (e != cudaSuccess) return cuda_fail(e, "nfsep pass 2");
  e = nfs::matvec_launch_mask<double>(a, 4);
  if (e != cudaSuccess) return cuda_fail(e, "nfsep pass 3");
  e = nfs::nfsep_post(c->Ap64, out, c->lam64, c->n1, c->n2, c->n3, v, sigma, s);
  if (e != cudaSuccess) return cuda_fail(e, "nfsep post");
  c->launches += 3 + 2 * nfs::plane_pass_kernels<double>(c->n1);
  return NFS_OK;
}

using nfs::host::cplxd;

// Long-vector operations of the Krylov drivers on device vectors (P = 1):
// basis V (vector j at V + j N) and work vector w, on the context's stream.
struct DevBasis : virtual nfs::host::KrylovOps {
  nfs_ctx* c;
  double2* V;
  double2* w;
  long long N;
  cudaStream_t s;
  DevBasis(nfs_ctx* ctx, double2* basis, double2* work) : c(ctx), V(basis), w(work), N(ctx->N), s(ctx->work) {}
  int put_coef(const std::vector<cplxd>& cf, double* dst) {
    for (size_t i = 0; i < cf.size(); ++i) {
      c->hscratch[2 * i] = cf[i].real();
      c->hscratch[2 * i + 1] = cf[i].imag();
    }
    CK(cudaMemcpyAsync(dst, c->hscratch, cf.size() * 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    return NFS_OK;
  }
  int dots(int m, std::vector<cplxd>& out) override {
    double* part = c->dscratch;
    double* fin = c->dscratch + (size_t)kRedBlocks * 2 * m;
    nfs::k_multi_dot<kRedThreads><<<dim3(kRedBlocks, 1), kRedThreads, 0, s>>>(V, 0, m, w, N, part, nullptr);
    nfs::k_multi_dot_finish<<<dim3(m, 1), kRedThreads, 0, s>>>(part, m, kRedBlocks, fin, nullptr);
    CK(cudaGetLastError());
    c->launches += 2;
    CK(cudaMemcpyAsync(c->hscratch, fin, (size_t)m * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out.resize(m);
    for (int i = 0; i < m; ++i) out[i] = cplxd(c->hscratch[2 * i], c->hscratch[2 * i + 1]);
    return NFS_OK;
  }
  int axpy(int m, const std::vector<cplxd>& cf) override {
    double* dc = c->dscratch;
    TRY(put_coef(cf, dc));
    CK(nfs::zaxpy_basis(w, V, N, dc, m, 1.0, s));
    c->launches += 1;
    CK(cudaStreamSynchronize(s));  // the pinned staging buffer is reused next
    return NFS_OK;
  }
  int norm(double& nrm) override {
    nfs::k_dot_re<double2><<<dim3(kRedBlocks, 1), kRedThreads, 0, s>>>(w, w, N, c->dscratch, kRedBlocks, nullptr, 0);
    CK(cudaGetLastError());
    c->launches += 1;
    CK(cudaMemcpyAsync(c->hscratch, c->dscratch, kRedBlocks * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double t = 0.0;
    for (int i = 0; i < kRedBlocks; ++i) t += c->hscratch[i];
    nrm = std::sqrt(std::max(t, 0.0));
    return NFS_OK;
  }
  int store(int j, double scale) override {
    CK(nfs::zscale_copy(w, V + (long long)j * N, scale, N, s));
    c->launches += 1;
    return NFS_OK;
  }
  int rotate(int m, const std::vector<cplxd>& Q, int k) override {
    const size_t need = (size_t)m * k * 2;
    if (c->zY_len < need) {
      if (c->zY) cudaFree(c->zY);
      c->zY = nullptr;
      TRY(dalloc(c, &c->zY, need));
      c->zY_len = need;
    }
    std::vector<double> h(need);
    for (size_t i = 0; i < Q.size(); ++i) {
      h[2 * i] = Q[i].real();
      h[2 * i + 1] = Q[i].imag();
    }
    CK(cudaMemcpyAsync(c->zY, h.data(), need * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(nfs::zrotate(V, m, c->zY, k, N, s));
    c->launches += 1;
    CK(cudaStreamSynchronize(s));  // h is released next
    return NFS_OK;
  }
  int copy(int dst, int src) override {
    CK(cudaMemcpyAsync(V + (long long)dst * N, V + (long long)src * N, N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    return NFS_OK;
  }
  int load(int j) override {
    CK(cudaMemcpyAsync(w, V + (long long)j * N, N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    return NFS_OK;
  }
  int random(unsigned long long seed) override {
    nfs::k_random_fill<<<grid_blocks(N, 256), 256, 0, s>>>(w, N, 0, 1, seed);
    CK(cudaGetLastError());
    c->launches += 1;
    return NFS_OK;
  }
};

// Scratch of the device GMRES (offsets in doubles into dscratch): the two
// Gram-Schmidt passes' partials, the norm partials, the least-squares
// solution, the GmresDev state, then gs_axpy's partial sums.
constexpr size_t kGsPartLen = (size_t)64 * nfs::kGmresMax * 2;
constexpr size_t kGsNrmLen = 152 * 16 + 128;
constexpr size_t kGsYOff = 2 * kGsPartLen + kGsNrmLen;
constexpr size_t kGsStateOff = kGsYOff + 2 * nfs::kGmresMax;
constexpr size_t kGsTmpOff = kGsStateOff + (sizeof(nfs::GmresDev) + 15) / 16 * 2;
static_assert(kGsYOff % 2 == 0 && kGsStateOff % 2 == 0 && kGsTmpOff % 2 == 0, "16-byte alignment");
size_t gs_scratch_len(long long N) { return kGsTmpOff + 2 * (size_t)nfs::gs_axpy_tmp_len(N); }
// steps enqueued between two host reads of the Hessenberg columns
constexpr int kGmresBatch = 10;

// Steps j0 .. j0 + nsteps - 1 of a GMRES cycle of length m on stream s:
// w = (M - sigma I) V_j, two classical Gram-Schmidt passes, column j of H,
// V_{j+1} = w / h_{j+1,j}.
int enqueue_gmres_steps(nfs_ctx* c, cudaStream_t s, double2 sigma, double2* V, double2* w, int m, int j0, int nsteps) {
  const long long N = c->N;
  double* part1 = c->dscratch;
  double* part2 = c->dscratch + kGsPartLen;
  double* nrm = c->dscratch + 2 * kGsPartLen;
  auto* st = reinterpret_cast<nfs::GmresDev*>(c->dscratch + kGsStateOff);
  auto* tmp = reinterpret_cast<double2*>(c->dscratch + kGsTmpOff);
  const int S = nfs::gs_chunks(N), nb = nfs::gs_norm_blocks(N);
  for (int j = j0; j < j0 + nsteps; ++j) {
    const double2* vj = V + (long long)j * N;
    TRY(nfsep_apply(c, s, vj, w, vj, sigma));
    CK(nfs::gs_dots(V, j + 1, w, N, part1, s));
    CK(nfs::gs_axpy(w, V, N, j + 1, part1, nullptr, tmp, s));
    CK(nfs::gs_dots(V, j + 1, w, N, part2, s));
    CK(nfs::gs_axpy(w, V, N, j + 1, part2, nrm, tmp, s));
    CK(nfs::gmres_column(j, part1, part2, S, nrm, nb, st, s));
    c->launches += 3 + 2 * nfs::gs_axpy_kernels(N);
    if (j + 1 < m) {
      CK(nfs::gmres_store(w, V + (long long)(j + 1) * N, st, N, s));
      c->launches += 1;
    }
  }
  return NFS_OK;
}

// The same steps as a CUDA graph, captured on first use per (j0, nsteps, m,
// buffers, shift) and replayed on later cycles and solves: one launch
// instead of about a dozen per step.  s must be the context's work stream
// (graph capture is not possible on the legacy default stream).
#ifndef NFS_GMRES_GRAPH
#define NFS_GMRES_GRAPH 1
#endif
int gmres_steps(nfs_ctx* c, cudaStream_t s, double2 sigma, double2* V, double2* w, int m, int j0, int nsteps) {
  if (!NFS_GMRES_GRAPH) return enqueue_gmres_steps(c, s, sigma, V, w, m, j0, nsteps);
  // one set of batches is kept: a new shift or buffer replaces it
  if (!c->gm_graphs.empty()) {
    const GmresGraph& f = c->gm_graphs.front();
    if (f.m != m || f.V != V || f.w != w || f.scratch != c->dscratch || f.sigma_re != sigma.x ||
        f.sigma_im != sigma.y) {
      for (GmresGraph& g : c->gm_graphs) cudaGraphExecDestroy(g.exec);
      c->gm_graphs.clear();
    }
  }
  for (const GmresGraph& g : c->gm_graphs)
    if (g.j0 == j0 && g.nsteps == nsteps) {
      CK(cudaGraphLaunch(g.exec, s));
      c->launches += g.kernels;
      return NFS_OK;
    }
  const long long l0 = c->launches;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_gmres_steps(c, s, sigma, V, w, m, j0, nsteps);
  cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  const long long kernels = c->launches - l0;
  c->launches = l0;
  if (rc != NFS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture (gmres)");
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (gmres)");
  c->gm_graphs.push_back(GmresGraph{j0, nsteps, m, V, w, c->dscratch, sigma.x, sigma.y, kernels, exec});
  CK(cudaGraphLaunch(exec, s));
  c->launches += kernels;
  return NFS_OK;
}

// Restarted GMRES(m) on (M - sigma I) x = b (x holds the start iterate), the
// iteration of nfs::host::gmres: the long-vector work on the device (V, m + 1
// vectors, and w as workspace), the least-squares problem on the host
// (GivensLS) from the Hessenberg columns read once per batch of kGmresBatch
// steps.  Steps enqueued after the one that converged are wasted work (the
// cycle ends at the converged column); they are counted as iterations.
int dev_gmres(nfs_ctx* c, const double2* b, double2* x, double2 sigma, double2* V, double2* w, int m, double tol,
              double bnorm, int maxit, nfs::host::GmresResult& out) {
  out = nfs::host::GmresResult{};
  if (m < 1 || m > nfs::kGmresMax || !(tol > 0.0)) return NFS_EINVAL;
  if (!(bnorm > 0.0)) return NFS_OK;
  cudaStream_t s = c->work;
  const long long N = c->N;
  double* nrm = c->dscratch + 2 * kGsPartLen;
  double* yd = c->dscratch + kGsYOff;
  auto* st = reinterpret_cast<nfs::GmresDev*>(c->dscratch + kGsStateOff);
  const int nb = nfs::gs_norm_blocks(N);
  const double tolb = tol * bnorm;
  constexpr int kCol = nfs::kGmresMax + 1;
  nfs::host::GivensLS ls;
  std::vector<nfs::host::cplxd> col(kCol), y;
  for (;;) {
    // r = b - (M - sigma I) x; V_0 = r / ||r||
    TRY(nfsep_apply(c, s, x, w, x, sigma));
    CK(nfs::gmres_residual(b, w, N, nrm, s));
    c->launches += 1;
    CK(cudaMemcpyAsync(c->hscratch, nrm, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double bb = 0.0;
    for (int i = 0; i < nb; ++i) bb += c->hscratch[i];
    const double beta = std::sqrt(std::max(bb, 0.0));
    out.relres = beta / bnorm;
    if (beta <= tolb) return NFS_OK;
    if (out.iterations >= maxit) {
      out.status = NFS_ENOCONV;
      return NFS_OK;
    }
    CK(cudaMemsetAsync(st, 0, 2 * sizeof(double2), s));  // done, inv_h
    CK(nfs::zscale_copy(w, V, 1.0 / beta, N, s));
    c->launches += 1;
    ls.reset(m, beta);
    int j = 0;
    bool done = false;
    while (j < m && out.iterations < maxit && !done) {
      const int steps = std::min({kGmresBatch, m - j, maxit - out.iterations});
      TRY(gmres_steps(c, s, sigma, V, w, m, j, steps));
      const auto* hc_dev = reinterpret_cast<const double2*>(reinterpret_cast<const char*>(st) +
                                                             offsetof(nfs::GmresDev, Hc));
      CK(cudaMemcpyAsync(c->hscratch, hc_dev + (size_t)j * kCol, (size_t)steps * kCol * sizeof(double2),
                         cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int t = 0; t < steps && !done; ++t) {
        const double* hc = c->hscratch + (size_t)t * kCol * 2;
        const int jj = j + t;
        for (int i = 0; i <= jj; ++i) col[i] = nfs::host::cplxd(hc[2 * i], hc[2 * i + 1]);
        const double h = hc[2 * (jj + 1)];
        const double res = ls.add_column(col.data(), h);
        done = res <= tolb || h == 0.0;
      }
      j += steps;
      out.iterations += steps;
    }
    // y = R^{-1} g over the cycle's columns, x += V y
    if (!ls.solve(y)) return NFS_EBREAKDOWN;
    for (size_t i = 0; i < y.size(); ++i) {
      c->hscratch[2 * i] = y[i].real();
      c->hscratch[2 * i + 1] = y[i].imag();
    }
    CK(cudaMemcpyAsync(yd, c->hscratch, y.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    CK(nfs::zaxpy_basis(x, V, N, yd, ls.columns(), -1.0, s));
    c->launches += 1;
    CK(cudaStreamSynchronize(s));  // the pinned staging buffer is reused next
    ++out.restarts;
  }
}

// Arnoldi on (M - sigma I)^{-1}: each application one GMRES solve
struct DevShiftInvert : DevBasis {
  double2* gV;  // GMRES basis
  double2* gw;  // GMRES work vector
  double2* gx;  // GMRES iterate
  double2 sigma;
  int gm;
  double tol;
  int maxit;
  long long inner = 0;
  DevShiftInvert(nfs_ctx* ctx, double2* basis, double2* work, double2* gbasis, double2* gwork, double2* gxv,
                 double2 sg, int m_inner, double t, int mi)
      : DevBasis(ctx, basis, work), gV(gbasis), gw(gwork), gx(gxv), sigma(sg), gm(m_inner), tol(t), maxit(mi) {}
  int apply(int j) override {
    CK(cudaMemsetAsync(gx, 0, N * sizeof(double2), s));
    nfs::host::GmresResult r;
    // the Arnoldi vectors have unit norm
    TRY(dev_gmres(c, V + (long long)j * N, gx, sigma, gV, gw, gm, tol, 1.0, maxit, r));
    inner += r.iterations;
    if (r.status != 0) return NFS_ENOCONV;
    CK(cudaMemcpyAsync(w, gx, N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    return NFS_OK;
  }
};

constexpr int kGmresRestart = 100;

int ensure_nfsep_bases(nfs_ctx* c, int m, int gm) {
  if (c->zv_cap < m + 1) {
    if (c->zv) cudaFree(c->zv);
    c->zv = nullptr;
    c->zv_cap = 0;
    TRY(dalloc(c, &c->zv, (size_t)(m + 1) * c->N));
    c->zv_cap = m + 1;
  }
  if (c->gv_cap < gm + 1) {
    if (c->gv) cudaFree(c->gv);
    c->gv = nullptr;
    c->gv_cap = 0;
    TRY(dalloc(c, &c->gv, (size_t)(gm + 1) * c->N));
    c->gv_cap = gm + 1;
  }
  return ensure_scratch(c, std::max(gs_scratch_len(c->N), (size_t)kRedBlocks * 2 * (std::max(m, gm) + 2) +
                                                               4 * (size_t)(std::max(m, gm) + 2) + 64));
}

// Arnoldi basis size of an NFSEP eigensolve for nev values (opt.ncv or
// max(2 nev + 2, 20), at most N - 1) and the GMRES restart length
int nfsep_sizes(const nfs_ctx* c, int nev, int& m, int& gm) {
  m = c->opt.ncv > 0 ? c->opt.ncv : std::max(2 * nev + 2, 20);
  m = (int)std::min<long long>(m, c->N - 1);
  if (m < nev + 2) return NFS_EINVAL;
  gm = (int)std::min<long long>(kGmresRestart, c->N - 1);
  return NFS_OK;
}

int nfsep_reserve(nfs_ctx* c, int nev) {
  int m = 0, gm = 0;
  TRY(nfsep_sizes(c, nev, m, gm));
  TRY(ensure_nfsep_bases(c, m, gm));
  // the Krylov-Schur restart rotation (at most m x m, interleaved complex)
  const size_t need = (size_t)m * m * 2;
  if (c->zY_len < need) {
    if (c->zY) cudaFree(c->zY);
    c->zY = nullptr;
    TRY(dalloc(c, &c->zY, need));
    c->zY_len = need;
  }
  return NFS_OK;
}

}  // namespace

extern "C" int nfs_setup_biiso(nfs_ctx** out, const int grid[3], const double* lattice, const double k[3],
                               const nfs_biiso_material* bm, const nfs_options* opt) {
  if (!out) return NFS_EINVAL;
  *out = nullptr;
  if (!grid || !k || !bm || !bm->eps || !bm->gamma) return NFS_EINVAL;
  for (int l = 0; l < 3; ++l)
    if (grid[l] <= 0) return NFS_EINVAL;
  const long long n = (long long)grid[0] * grid[1] * grid[2];
  // B^{-1} per voxel and component (eq. mtx_B): B_c = i [[zeta, mu], [-eps, -xi]],
  // xi = chi + i gamma, zeta = chi - i gamma; det B_c = zeta xi - mu eps
  std::vector<double2> binv((size_t)12 * n);
  for (int cpt = 0; cpt < 3; ++cpt)
    for (long long v = 0; v < n; ++v) {
      const size_t i = (size_t)cpt * n + v;
      auto cx = [&](const double* a, cplxd dflt) { return a ? cplxd(a[2 * i], a[2 * i + 1]) : dflt; };
      const cplxd eps = cx(bm->eps, 1.0), mu = cx(bm->mu, 1.0), gam = cx(bm->gamma, 0.0), chi = cx(bm->chi, 0.0);
      const cplxd I(0.0, 1.0);
      const cplxd xi = chi + I * gam, zeta = chi - I * gam;
      const cplxd det = zeta * xi - mu * eps;
      const double scale = std::abs(zeta) * std::abs(xi) + std::abs(mu) * std::abs(eps);
      if (!std::isfinite(std::abs(det)) || !(std::abs(det) > 1e-12 * scale)) return NFS_EINVAL;
      const cplxd inv[4] = {-I * xi / det, -I * mu / det, I * eps / det, I * zeta / det};
      for (int t = 0; t < 4; ++t) binv[(size_t)(4 * cpt + t) * n + v] = make_double2(inv[t].real(), inv[t].imag());
    }
  // the product's tables come from the ordinary set-up with a placeholder
  // chiral medium (eps = 1, gamma = 0), whose material arrays stay unused
  std::vector<double> ones((size_t)3 * n, 1.0), zeros((size_t)3 * n, 0.0);
  nfs_material placeholder{};
  placeholder.kind = NFS_MEDIUM_CHIRAL;
  placeholder.axis_a = 0;
  placeholder.axis_b = 1;
  placeholder.eps = ones.data();
  placeholder.mu = nullptr;
  placeholder.gamma = zeros.data();
  nfs_ctx* c = nullptr;
  TRY(nfs_setup(&c, grid, lattice, k, &placeholder, opt));
  const int rc = [&]() -> int {
    TRY(dalloc(c, &c->binv64, binv.size()));
    CK(cudaMemcpy(c->binv64, binv.data(), binv.size() * sizeof(double2), cudaMemcpyHostToDevice));
    CK(nfs::nfsep_prepare(c->n3));
    return NFS_OK;
  }();
  if (rc != NFS_OK) {
    nfs_destroy(c);
    return rc;
  }
  *out = c;
  return NFS_OK;
}

extern "C" int nfs_nfsep_matvec(nfs_ctx* c, const void* y, void* My) {
  if (!c || !y || !My || y == My) return NFS_EINVAL;
  if (!c->binv64) return NFS_EUNSUPPORTED;
  if (((uintptr_t)y | (uintptr_t)My) & 15) return NFS_EINVAL;
  return nfsep_apply(c, c->stream, (const double2*)y, (double2*)My, nullptr, make_double2(0.0, 0.0));
}

extern "C" int nfs_nfsep_eigs(nfs_ctx* c, int nev, const double sigma[2], double* omega, void* Y,
                              nfs_nfsep_info* info) {
  if (!c || !sigma || !omega || nev <= 0) return NFS_EINVAL;
  if (!c->binv64) return NFS_EUNSUPPORTED;
  if (!(std::isfinite(sigma[0]) && std::isfinite(sigma[1]))) return NFS_EINVAL;
  int m = 0, gm = 0;
  TRY(nfsep_sizes(c, nev, m, gm));
  TRY(ensure_nfsep_bases(c, m, gm));
  const double2 sg = make_double2(sigma[0], sigma[1]);
  const long long launches_0 = c->launches;
  // everything below runs on the work stream (the GMRES step batches are
  // captured as graphs), ordered after the caller's stream
  TRY(join_caller(c));
  // start vector
  nfs::k_random_fill<<<grid_blocks(c->N, 256), 256, 0, c->work>>>(c->zv, c->N, 0, 1, c->opt.seed);
  CK(cudaGetLastError());
  c->launches += 1;
  DevShiftInvert op(c, c->zv, c->p64, c->gv, c->r64, c->x64, sg, gm, c->opt.cg_tol, c->opt.cg_maxit);
  nfs::host::ArnoldiResult r;
  const int rc = nfs::host::krylov_schur(op, nev, m, c->opt.eig_tol, c->opt.max_restarts, r);
  if (rc != NFS_OK) {
    // an inner solve failed (or a breakdown): nothing to return but the counts
    if (info) {
      *info = nfs_nfsep_info{};
      info->arnoldi_steps = r.steps;
      info->restarts = r.restarts;
      info->gmres_iterations = op.inner;
      info->status = rc;
      info->kernel_launches = c->launches - launches_0;
    }
    return rc;
  }
  for (int e = 0; e < nev; ++e) {
    const cplxd lam = cplxd(sigma[0], sigma[1]) + 1.0 / r.theta[e];
    omega[2 * e] = lam.real();
    omega[2 * e + 1] = lam.imag();
  }
  if (Y) CK(cudaMemcpyAsync(Y, c->zv, (size_t)nev * c->N * sizeof(double2), cudaMemcpyDeviceToDevice, c->work));
  CK(cudaStreamSynchronize(c->work));
  if (info) {
    info->arnoldi_steps = r.steps;
    info->restarts = r.restarts;
    info->gmres_iterations = op.inner;
    info->nconv = r.nconv;
    info->max_ritz_residual = r.max_residual;
    info->status = r.status;
    info->kernel_launches = c->launches - launches_0;
  }
  return r.status;
}

extern "C" int nfs_nfsep_fields(nfs_ctx* c, int m, const void* Yv, void* Xv) {
  if (!c || m <= 0 || !Yv || !Xv) return NFS_EINVAL;
  if (!c->binv64) return NFS_EUNSUPPORTED;
  if ((((uintptr_t)Yv) | ((uintptr_t)Xv)) & 15) return NFS_EINVAL;
  const long long n = c->n, N = c->N;
  for (int j = 0; j < m; ++j) {
    // Algorithm 1, second branch: y <- Sigma^{1/2} y, x = B^{-1} diag(P_r, Q_r) y
    cudaError_t e = nfs::nfsep_prescale((const double2*)Yv + (long long)j * N, c->t64, c->lam64, c->n1, c->n2,
                                        c->n3, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "nfsep fields prescale");
    nfs::MatvecArgs<double> a = margs<double>(c, c->t64, nullptr, nullptr);
    e = nfs::pass1_launch<double>(a);
    if (e != cudaSuccess) return cuda_fail(e, "nfsep fields pass 1");
    e = nfs::nfsep_fields((const double2*)c->fld, c->binv64, c->tw64[2], c->bloch64, c->n1, c->n2, c->n3,
                          (double2*)Xv + (long long)j * 6 * n, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "nfsep fields");
    c->launches += 2 + nfs::plane_pass_kernels<double>(c->n1);
  }
  return NFS_OK;
}

// --- batches -------------------------------------------------------------------

extern "C" int nfs_setup_batch(nfs_batch** out, int nprob, const nfs_problem* probs, const nfs_options* opt) {
  if (!out) return NFS_EINVAL;
  *out = nullptr;
  if (nprob <= 0 || !probs) return NFS_EINVAL;
  const nfs_options o = resolved_options(opt);
  TRY(check_options(o));
  // group by (grid, medium kind, axis pair, mu present)
  std::map<std::tuple<int, int, int, int, int, int, int>, std::vector<int>> groups;
  for (int i = 0; i < nprob; ++i) {
    const nfs_problem& p = probs[i];
    const int ax_a = p.mat.kind == NFS_MEDIUM_PSEUDOCHIRAL ? p.mat.axis_a : 0;
    const int ax_b = p.mat.kind == NFS_MEDIUM_PSEUDOCHIRAL ? p.mat.axis_b : 1;
    groups[std::make_tuple(p.grid[0], p.grid[1], p.grid[2], p.mat.kind, ax_a, ax_b, p.mat.mu != nullptr ? 1 : 0)]
        .push_back(i);
  }
  // every problem is validated on the host before any device memory is taken
  struct ClassPrep {
    std::vector<int> ids;
    std::vector<const nfs_material*> ms;
    std::vector<Prepared> prep;
    double delta[3];
  };
  std::vector<ClassPrep> cls;
  for (auto& kv : groups) {
    ClassPrep cp;
    cp.ids = kv.second;
    const int P = (int)cp.ids.size();
    std::vector<const double*> lat(P, nullptr), ks(P);
    cp.ms.resize(P);
    for (int q = 0; q < P; ++q) {
      ks[q] = probs[cp.ids[q]].k;
      cp.ms[q] = &probs[cp.ids[q]].mat;
    }
    TRY(prepare_class(P, probs[cp.ids[0]].grid, lat.data(), ks.data(), cp.ms.data(), o, cp.prep, cp.delta));
    cls.push_back(std::move(cp));
  }
  nfs_batch* b = new (std::nothrow) nfs_batch();
  if (!b) return NFS_ENOMEM;
  b->where.assign(nprob, std::make_pair(-1, -1));
  for (ClassPrep& cp : cls) {
    const std::vector<int>& ids = cp.ids;
    const int P = (int)ids.size();
    nfs_ctx* c = nullptr;
    const int rc = setup_class(&c, P, probs[ids[0]].grid, cp.ms.data(), cp.prep, cp.delta, o);
    std::vector<Prepared>().swap(cp.prep);
    if (rc != NFS_OK) {
      nfs_destroy_batch(b);
      return rc;
    }
    for (int q = 0; q < P; ++q) b->where[ids[q]] = std::make_pair((int)b->classes.size(), q);
    b->classes.push_back(c);
  }
  *out = b;
  return NFS_OK;
}

extern "C" int nfs_eigs_batch(nfs_batch* b, int nev, double* omega, nfs_eigs_info* info) {
  if (!b || !omega || nev <= 0) return NFS_EINVAL;
  const int nc = (int)b->classes.size();
  std::vector<std::vector<double>> om(nc);
  std::vector<std::vector<nfs_eigs_info>> inf(nc);
  std::vector<int> rc(nc, NFS_OK);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  for (int i = 0; i < nc; ++i) {
    nfs_ctx* c = b->classes[i];
    if (nev >= c->N / 2) return NFS_EINVAL;
    om[i].assign((size_t)c->P * nev, 0.0);
    inf[i].assign(c->P, nfs_eigs_info{});
    TRY(join_caller(c));
  }
  // the classes run concurrently: one basis size for all, within 80% of the
  // free device memory together, and the bases allocated here, in turn
  // (restarts cost accuracy as well as time: each assumes the Lanczos relation
  // of the inexact solves to hold exactly)
  if (b->classes[0]->opt.ncv <= 0) {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    double per = 0.0;
    for (nfs_ctx* c : b->classes) per += basis_bytes_per_vector(c);
    int m = std::min(wanted_ncv(nev), (int)std::max(0.0, 0.8 * (double)fr / per) - 1);
    m = std::max(m, 2 * nev + 2);
    for (nfs_ctx* c : b->classes) {
      c->ncv_set = (int)std::min<long long>(m, c->N - 1);
      TRY(ensure_basis(c, c->ncv_set));
    }
  }
  // one host thread per grid class; each drives its own stream
  std::vector<std::thread> th;
  for (int i = 0; i < nc; ++i)
    th.emplace_back([&, i]() {
      cudaSetDevice(dev);
      rc[i] = eigs_core(b->classes[i], nev, om[i].data(), nullptr, inf[i].data());
    });
  for (auto& t : th) t.join();
  int worst = NFS_OK;
  for (int i = 0; i < nc; ++i)
    if (rc[i] != NFS_OK && (worst == NFS_OK || rc[i] != NFS_ENOCONV)) worst = rc[i];
  if (worst != NFS_OK && worst != NFS_ENOCONV) return worst;
  const int nprob = (int)b->where.size();
  for (int pi = 0; pi < nprob; ++pi) {
    const int ci = b->where[pi].first, q = b->where[pi].second;
    std::copy(om[ci].begin() + (size_t)q * nev, om[ci].begin() + (size_t)(q + 1) * nev, omega + (size_t)pi * nev);
    if (info) info[pi] = inf[ci][q];
  }
  return worst;
}

extern "C" int nfs_band_structure(const int grid[3], const nfs_material* mat, int nk, const double* k,
                                  const nfs_options* opt, int nev, int max_chunk, double* omega,
                                  nfs_eigs_info* info, int* chunks) {
  if (!grid || !mat || nk <= 0 || !k || nev <= 0 || !omega) return NFS_EINVAL;
  const nfs_options o = resolved_options(opt);
  TRY(check_options(o));
  for (int l = 0; l < 3; ++l)
    if (grid[l] <= 0) return NFS_EINVAL;
  const double n = (double)grid[0] * grid[1] * grid[2];
  // device bytes one k-point needs: its Lanczos basis at the full size (the
  // same basis size nfs_eigs_batch would choose with room to spare: no
  // restarts) and the fixed workspaces of a context (material copies, basis
  // tables, fields, six complex128 and four complex64 vectors), rounded up
  const int m = o.ncv > 0 ? o.ncv : wanted_ncv(nev);
  const double per_k = (double)(m + 1) * 4.0 * n * (16 + 16 + 8 + 8 + 8) + 1024.0 * n;
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  int chunk = (int)std::min<double>(nk, std::max(1.0, std::floor(0.8 * (double)fr / per_k)));
  if (max_chunk > 0) chunk = std::min(chunk, max_chunk);
  int nchunks = 0, worst = NFS_OK;
  std::vector<nfs_problem> probs;
  for (int k0 = 0; k0 < nk; k0 += chunk) {
    const int P = std::min(chunk, nk - k0);
    probs.assign(P, nfs_problem{});
    for (int q = 0; q < P; ++q) {
      for (int l = 0; l < 3; ++l) {
        probs[q].grid[l] = grid[l];
        probs[q].k[l] = k[3 * (size_t)(k0 + q) + l];
      }
      probs[q].mat = *mat;
    }
    nfs_batch* b = nullptr;
    TRY(nfs_setup_batch(&b, P, probs.data(), &o));
    const int rc = nfs_eigs_batch(b, nev, omega + (size_t)k0 * nev, info ? info + k0 : nullptr);
    nfs_destroy_batch(b);
    ++nchunks;
    if (rc != NFS_OK && rc != NFS_ENOCONV) return rc;
    if (rc == NFS_ENOCONV) worst = rc;
  }
  if (chunks) *chunks = nchunks;
  return worst;
}

extern "C" int nfs_batch_num_classes(const nfs_batch* b) { return b ? (int)b->classes.size() : 0; }

extern "C" void nfs_destroy_batch(nfs_batch* b) {
  if (!b) return;
  for (nfs_ctx* c : b->classes) nfs_destroy(c);
  delete b;
}
