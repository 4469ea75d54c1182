// nfs_matvec_noalloc: the A_r product for callers that cannot allocate
// device memory.  Some host applications own every byte of the GPU: a
// framework that reserved the device through its own caching allocator (where
// a raw cudaMalloc can fail or fragment its pool), or a service with a fixed
// device-memory budget that must not allocate after start-up.  For them this
// entry point takes its workspace from a fixed, file-scope device array
// instead of nfs_setup's allocations; the caller still passes every input
// and output.
//
// The array below is created when the library's device code is loaded and is
// held by every GPU that loads it until the process exits.  In host code its
// name is only a stand-in: its device address is obtained per device with
// cudaGetSymbolAddress on the first call on that device (with that device
// current) and passed to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/nfs.h"
#include "matvec.h"

namespace {

constexpr long long kMaxVoxels = NFS_NOALLOC_MAX_VOXELS;
constexpr int kMaxEdge = 128;
constexpr int kMaxDevices = 64;

// Layout of the scratch array (offsets in bytes, each 256-aligned):
//   fields   6 n complex128         (the three passes' workspace)
//   inv_phi  3 n double             (1 / Phi per component)
//   gamma    3 n double             (chiral: per component; pseudochiral: first n)
//   lambda   3 * kMaxEdge complex128 (Lambda_1 | Lambda_2 | Lambda_3)
//   twiddle  3 * kMaxEdge complex128 (exp(-2 pi i m / n_l) per axis)
//   status   int                    (1: Phi <= 0 somewhere; 2: eps or gamma not finite)
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffFld = 0;
constexpr size_t kOffPhi = align256(kOffFld + 6 * kMaxVoxels * sizeof(double2));
constexpr size_t kOffGam = align256(kOffPhi + 3 * kMaxVoxels * sizeof(double));
constexpr size_t kOffLam = align256(kOffGam + 3 * kMaxVoxels * sizeof(double));
constexpr size_t kOffTw = align256(kOffLam + 3 * kMaxEdge * sizeof(double2));
constexpr size_t kOffStatus = align256(kOffTw + 3 * kMaxEdge * sizeof(double2));
constexpr size_t kScratchBytes = align256(kOffStatus + sizeof(int));
static_assert(kScratchBytes == 4731136, "the workspace size documented in nfs.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

struct Tables {
  double2* lam;
  double2* tw;
  double* inv_phi;
  double* gam;
  int* status;
};

// Lambda_l[i] = (exp(i 2 pi (i + k.a_l)/n_l) - 1) / delta_l with the real part
// written as -2 sin^2(pi (i + k.a_l)/n_l); twiddles exp(-2 pi i m / n_l);
// 1/Phi and gamma from the caller's eps and gamma (mu = 1).
__global__ void k_noalloc_prep(Tables t, const double* __restrict__ eps, const double* __restrict__ gamma, int n1,
                               int n2, int n3, double k1, double k2, double k3, double d1, double d2, double d3,
                               int kind, int ax_a, int ax_b) {
  const long long n = (long long)n1 * n2 * n3;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int nl[3] = {n1, n2, n3};
  const double kl[3] = {k1, k2, k3};
  const double dl[3] = {d1, d2, d3};
  for (long long i = tid; i < 3 * kMaxEdge; i += stride) {
    const int l = (int)(i / kMaxEdge), m = (int)(i % kMaxEdge);
    if (m < nl[l]) {
      const double x = (m + kl[l]) / nl[l];
      const double sh = sinpi(x);
      t.lam[(l == 0 ? 0 : l == 1 ? n1 : n1 + n2) + m] = make_double2(-2.0 * sh * sh / dl[l], sinpi(2.0 * x) / dl[l]);
      double s, c;
      sincospi(-2.0 * (double)m / nl[l], &s, &c);
      t.tw[l * kMaxEdge + m] = make_double2(c, s);
    }
  }
  for (long long v = tid; v < n; v += stride) {
    for (int c = 0; c < 3; ++c) {
      const double e = eps[c * n + v];
      double g, phi;
      if (kind == NFS_MEDIUM_CHIRAL) {
        g = gamma[c * n + v];
        phi = e - g * g;
        t.gam[c * n + v] = g;
      } else {
        g = gamma[v];
        phi = (c == ax_a || c == ax_b) ? e - g * g : e;
        if (c == 0) t.gam[v] = g;
      }
      // a non-finite eps or gamma is a bad argument (NFS_EINVAL, as nfs_setup
      // returns); otherwise Phi must be positive (NFS_ENOTHPD)
      if (!isfinite(e) || !isfinite(g)) {
        atomicMax(t.status, 2);
      } else if (!(phi > 0.0)) {
        atomicMax(t.status, 1);
      }
      t.inv_phi[c * n + v] = 1.0 / phi;
    }
  }
}

bool edge_ok(int s) {
  switch (s) {
    case 8: case 12: case 16: case 24: case 32: case 48: case 64: case 96: case 128: return true;
    default: return false;
  }
}

}  // namespace

extern "C" int nfs_matvec_noalloc(const int grid[3], const double k[3], int kind, int axis_a, int axis_b,
                                  const double* eps, const double* gamma, double alpha, double beta,
                                  const void* u, void* Au, void* stream) {
  if (!grid || !k || !eps || !gamma || !u || !Au || u == Au) return NFS_EINVAL;
  const int n1 = grid[0], n2 = grid[1], n3 = grid[2];
  if (!edge_ok(n1) || !edge_ok(n2) || !edge_ok(n3) || n1 != n2) return NFS_EUNSUPPORTED;
  const long long n = (long long)n1 * n2 * n3;
  if (n > kMaxVoxels) return NFS_EUNSUPPORTED;  // the static workspace holds 32^3 voxels at most
  if (!nfs::matvec_supported<double>(n1, n2, n3)) return NFS_EUNSUPPORTED;
  if (kind != NFS_MEDIUM_CHIRAL && kind != NFS_MEDIUM_PSEUDOCHIRAL) return NFS_EINVAL;
  if (kind == NFS_MEDIUM_PSEUDOCHIRAL &&
      (axis_a < 0 || axis_a > 2 || axis_b < 0 || axis_b > 2 || axis_a == axis_b))
    return NFS_EINVAL;
  if (alpha == 0.0 || beta == 0.0) return NFS_EBASIS;
  // the Lemma, checked on the host: Lambda_q > 0 and Lambda_p != 0 everywhere
  double lre[3][kMaxEdge], lim[3][kMaxEdge];
  const int nl[3] = {n1, n2, n3};
  bool all_int = true;
  for (int l = 0; l < 3; ++l) {
    if (!std::isfinite(k[l])) return NFS_EINVAL;
    if (std::fabs(k[l] - std::round(k[l])) > 1e-12) all_int = false;
    for (int m = 0; m < nl[l]; ++m) {
      const double th = 2.0 * M_PI * (m + k[l]) / nl[l];
      const double sh = std::sin(0.5 * th);
      lre[l][m] = -2.0 * sh * sh * nl[l];
      lim[l][m] = std::sin(th) * nl[l];
    }
  }
  if (all_int) return NFS_EKPOINT;
  for (int i3 = 0; i3 < n3; ++i3)
    for (int i2 = 0; i2 < n2; ++i2)
      for (int i1 = 0; i1 < n1; ++i1) {
        const double ar[3] = {lre[0][i1], lre[1][i2], lre[2][i3]}, ai[3] = {lim[0][i1], lim[1][i2], lim[2][i3]};
        const double lq = ar[0] * ar[0] + ai[0] * ai[0] + ar[1] * ar[1] + ai[1] * ai[1] + ar[2] * ar[2] + ai[2] * ai[2];
        const double pr[3] = {beta * ar[2] - ar[1], ar[0] - alpha * ar[2], alpha * ar[1] - beta * ar[0]};
        const double pi[3] = {beta * ai[2] - ai[1], ai[0] - alpha * ai[2], alpha * ai[1] - beta * ai[0]};
        const double lp = pr[0] * pr[0] + pi[0] * pi[0] + pr[1] * pr[1] + pi[1] * pi[1] + pr[2] * pr[2] + pi[2] * pi[2];
        if (!(lq > 0)) return NFS_EKPOINT;
        if (!(lp > 1e-13 * (alpha * alpha + beta * beta + 1.0) * lq)) return NFS_EBASIS;
      }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NFS_ECUDA;
  void* base = nullptr;
  {
    // one-time set-up per device, with that device current
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return NFS_ECUDA;
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
    // opt the kernels for this grid in to their shared memory (allocates nothing)
    e = nfs::matvec_prepare<double>(n1, n2, n3);
    if (e != cudaSuccess) return NFS_ECUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  Tables t;
  t.lam = reinterpret_cast<double2*>(b + kOffLam);
  t.tw = reinterpret_cast<double2*>(b + kOffTw);
  t.inv_phi = reinterpret_cast<double*>(b + kOffPhi);
  t.gam = reinterpret_cast<double*>(b + kOffGam);
  t.status = reinterpret_cast<int*>(b + kOffStatus);
  cudaStream_t s = (cudaStream_t)stream;
  // the status word keeps the previous call's value: clear it first
  e = cudaMemsetAsync(t.status, 0, sizeof(int), s);
  if (e != cudaSuccess) return NFS_ECUDA;
  const int threads = 256;
  const int blocks = (int)std::min<long long>((n + threads - 1) / threads + 2, 1024);
  k_noalloc_prep<<<blocks, threads, 0, s>>>(t, eps, gamma, n1, n2, n3, k[0], k[1], k[2], 1.0 / n1, 1.0 / n2,
                                            1.0 / n3, kind, axis_a, axis_b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return NFS_ECUDA;
  nfs::MatvecArgs<double> a{};
  a.u = static_cast<const double2*>(u);
  a.Au = static_cast<double2*>(Au);
  a.fld = reinterpret_cast<double2*>(b + kOffFld);
  a.lam = t.lam;
  a.tw1 = t.tw;
  a.tw2 = t.tw + kMaxEdge;
  a.tw3 = t.tw + 2 * kMaxEdge;
  a.inv_phi = t.inv_phi;
  a.gam = t.gam;
  a.inv_mu = nullptr;
  a.kind = kind;
  a.ax_a = kind == NFS_MEDIUM_CHIRAL ? 0 : axis_a;
  a.ax_b = kind == NFS_MEDIUM_CHIRAL ? 1 : axis_b;
  a.n1 = n1;
  a.n2 = n2;
  a.n3 = n3;
  a.alpha = alpha;
  a.beta = beta;
  a.skip = nullptr;
  a.stream = s;
  e = nfs::matvec_launch<double>(a);
  if (e != cudaSuccess) return NFS_ECUDA;
  int status = 0;
  e = cudaMemcpyAsync(&status, t.status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return NFS_ECUDA;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return NFS_ECUDA;
  return status == 2 ? NFS_EINVAL : (status ? NFS_ENOTHPD : NFS_OK);
}
