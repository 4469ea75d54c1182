// Vector kernels of the CG and Lanczos loops (Section 4.2: CG on A_r u = b;
// invert Lanczos on (B_r, A_r)).  Reductions are deterministic: a fixed grid
// of kRedBlocks blocks writes one partial per block, and a one-block kernel
// sums the partials in a fixed order.  Every CG kernel reads the device
// `done` flag first and returns at once when it is set, so a batch of
// launched iterations past convergence costs only empty launches.
#pragma once
#include <cstdint>

#include "nfs_complex.cuh"

namespace nfs {

constexpr int kRedBlocks = 304;   // two blocks per SM on a 152-SM GB300
constexpr int kRedThreads = 256;

// CG scalar state, device resident.
struct CGState {
  double rr;        // r^* r of the current residual
  double pAp;       // p^* A p
  double alpha, beta;
  double tol2;      // stop when rr <= tol2
  int it, maxit;
  int done;         // 1: converged, broken down or out of iterations
  int status;       // 0, -6 (no convergence) or -7 (breakdown)
  double part_a[kRedBlocks];
  double part_b[kRedBlocks];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[NT / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < NT / 32 ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ double sum_partials(const double* part) {
  // one block of kRedThreads threads sums kRedBlocks partials in fixed order
  double v = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) v += part[i];
  return block_sum<kRedThreads>(v);
}

// part[b] = sum over block b of Re(conj(x) y)
template <typename C>
__global__ void __launch_bounds__(kRedThreads)
k_dot_re(const C* __restrict__ x, const C* __restrict__ y, long long N, double* __restrict__ part,
         const int* __restrict__ skip) {
  if (skip && *skip) return;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kRedThreads) {
    const C a = x[i], b = y[i];
    acc += (double)a.x * (double)b.x + (double)a.y * (double)b.y;
  }
  const double s = block_sum<kRedThreads>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// CG start: rr = sum part_a; stop once r^* r <= tol2 (absolute threshold).
__global__ void __launch_bounds__(kRedThreads) k_cg_init(CGState* st, double tol2, int maxit) {
  const double rr = sum_partials(st->part_a);
  if (threadIdx.x == 0) {
    st->rr = rr;
    st->tol2 = tol2;
    st->it = 0;
    st->maxit = maxit;
    st->status = 0;
    st->alpha = st->beta = 0.0;
    st->done = (rr <= tol2) ? 1 : 0;
    if (!(rr == rr)) { st->done = 1; st->status = -7; }
  }
}

__global__ void __launch_bounds__(kRedThreads) k_cg_alpha(CGState* st) {
  if (st->done) return;
  const double pAp = sum_partials(st->part_a);
  if (threadIdx.x == 0) {
    st->pAp = pAp;
    if (!(pAp > 0.0)) {  // also catches NaN
      st->status = -7;
      st->done = 1;
    } else {
      st->alpha = st->rr / pAp;
    }
  }
}

// x += alpha p ; r -= alpha Ap ; part_b[block] = partial r^* r
template <typename C>
__global__ void __launch_bounds__(kRedThreads)
k_cg_update_xr(C* __restrict__ x, C* __restrict__ r, const C* __restrict__ p, const C* __restrict__ Ap, long long N,
               CGState* st) {
  if (st->done) return;
  using R = typename RealOf<C>::type;
  const R al = (R)st->alpha;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kRedThreads) {
    const C pi = p[i], api = Ap[i];
    C xi = x[i], ri = r[i];
    xi.x += al * pi.x;
    xi.y += al * pi.y;
    ri.x -= al * api.x;
    ri.y -= al * api.y;
    x[i] = xi;
    r[i] = ri;
    acc += (double)ri.x * (double)ri.x + (double)ri.y * (double)ri.y;
  }
  const double s = block_sum<kRedThreads>(acc);
  if (threadIdx.x == 0) st->part_b[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads) k_cg_beta(CGState* st) {
  if (st->done) return;
  const double rr = sum_partials(st->part_b);
  if (threadIdx.x == 0) {
    st->it += 1;
    if (!(rr == rr)) {
      st->status = -7;
      st->done = 1;
    } else if (rr <= st->tol2) {
      st->done = 1;
    } else if (st->it >= st->maxit) {
      st->status = -6;
      st->done = 1;
    }
    st->beta = rr / st->rr;
    st->rr = rr;
  }
}

// p = r + beta p
template <typename C>
__global__ void __launch_bounds__(kRedThreads)
k_cg_update_p(C* __restrict__ p, const C* __restrict__ r, long long N, CGState* st) {
  if (st->done) return;
  using R = typename RealOf<C>::type;
  const R be = (R)st->beta;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kRedThreads) {
    const C ri = r[i];
    C pi = p[i];
    pi.x = ri.x + be * pi.x;
    pi.y = ri.y + be * pi.y;
    p[i] = pi;
  }
}

// ---------------------------------------------------------------------------
// Elementwise helpers
// ---------------------------------------------------------------------------

// y = a - b
template <typename C>
__global__ void k_sub(const C* __restrict__ a, const C* __restrict__ b, C* __restrict__ y, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    y[i] = csub(a[i], b[i]);
}

// complex64 <- complex128 * s
__global__ void k_demote(const double2* __restrict__ a, double s, float2* __restrict__ y, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = a[i];
    y[i] = make_float2((float)(v.x * s), (float)(v.y * s));
  }
}

// x += s * complex128(d)
__global__ void k_axpy_promote(double2* __restrict__ x, double s, const float2* __restrict__ d, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = d[i];
    double2 xi = x[i];
    xi.x += s * (double)v.x;
    xi.y += s * (double)v.y;
    x[i] = xi;
  }
}

template <typename C>
__global__ void k_scale(C* __restrict__ a, double s, long long N) {
  using R = typename RealOf<C>::type;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    a[i] = cscale(a[i], (R)s);
}

// B_r v = i [Sigma^{-1} v2 ; -Sigma^{-1} v1], Sigma_r = diag(sqrt(Lq), sqrt(Lq))
// (eq. NFSEP_spd_1).  lam holds Lambda_1 | Lambda_2 | Lambda_3.
__global__ void k_apply_Br(const double2* __restrict__ v, double2* __restrict__ out, const double2* __restrict__ lam,
                           int n1, int n2, int n3) {
  const long long n = (long long)n1 * n2 * n3;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i1 = (int)(e % n1);
    const int i2 = (int)((e / n1) % n2);
    const int i3 = (int)(e / ((long long)n1 * n2));
    const double lq = cabs2(lam[i1]) + cabs2(lam[n1 + i2]) + cabs2(lam[n1 + n2 + i3]);
    const double is = 1.0 / sqrt(lq);
    const double2 v1a = v[e], v1b = v[n + e], v2a = v[2 * n + e], v2b = v[3 * n + e];
    out[e] = cmul_i(cscale(v2a, is));
    out[n + e] = cmul_i(cscale(v2b, is));
    out[2 * n + e] = cmul_mi(cscale(v1a, is));
    out[3 * n + e] = cmul_mi(cscale(v1b, is));
  }
}

// Counter-based uniform numbers in [-1, 1) (splitmix64 finaliser of the
// element index and seed): the Lanczos starting vector.
__device__ __forceinline__ double u01_hash(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

__global__ void k_random_fill(double2* __restrict__ v, long long N, unsigned long long seed) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long k = (unsigned long long)i * 2ull + seed * 0x632BE59BD9B4E019ull;
    v[i] = make_double2(u01_hash(k), u01_hash(k + 1));
  }
}

// ---------------------------------------------------------------------------
// Lanczos: basis stored contiguously, vector j at V + j * N (complex128).
// ---------------------------------------------------------------------------

// part[(b * m + j) * 2 + {0,1}] = block b's share of conj(V_j)^T w, j < m
template <int NT>
__global__ void __launch_bounds__(NT)
k_multi_dot(const double2* __restrict__ V, int m, const double2* __restrict__ w, long long N, double* __restrict__ part) {
  constexpr int EPT = 4;  // elements of w kept in registers per thread and pass
  for (int j0 = 0; j0 < m; ++j0) {
    double re = 0.0, im = 0.0;
    for (long long base = (long long)blockIdx.x * NT * EPT; base < N; base += (long long)gridDim.x * NT * EPT) {
#pragma unroll
      for (int t = 0; t < EPT; ++t) {
        const long long i = base + (long long)t * NT + threadIdx.x;
        if (i < N) {
          const double2 a = V[(long long)j0 * N + i], b = w[i];
          re += a.x * b.x + a.y * b.y;
          im += a.x * b.y - a.y * b.x;
        }
      }
    }
    re = block_sum<NT>(re);
    im = block_sum<NT>(im);
    if (threadIdx.x == 0) {
      part[((long long)blockIdx.x * m + j0) * 2 + 0] = re;
      part[((long long)blockIdx.x * m + j0) * 2 + 1] = im;
    }
  }
}

// out[j] = sum over nb blocks of part[b][j]  (one block per j)
__global__ void __launch_bounds__(kRedThreads)
k_multi_dot_finish(const double* __restrict__ part, int m, int nb, double* __restrict__ out) {
  const int j = blockIdx.x;
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nb; b += kRedThreads) {
    re += part[((long long)b * m + j) * 2 + 0];
    im += part[((long long)b * m + j) * 2 + 1];
  }
  re = block_sum<kRedThreads>(re);
  im = block_sum<kRedThreads>(im);
  if (threadIdx.x == 0) {
    out[2 * j] = re;
    out[2 * j + 1] = im;
  }
}

// w -= sum_j c_j V_j ; Mw -= sum_j c_j MV_j  (c complex, m entries)
__global__ void k_multi_axpy(double2* __restrict__ w, double2* __restrict__ Mw, const double2* __restrict__ V,
                             const double2* __restrict__ MV, const double* __restrict__ c, int m, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double2 a = w[i], b = Mw[i];
    for (int j = 0; j < m; ++j) {
      const double2 cj = make_double2(c[2 * j], c[2 * j + 1]);
      const double2 v = V[(long long)j * N + i], mv = MV[(long long)j * N + i];
      a = csub(a, cmul(cj, v));
      b = csub(b, cmul(cj, mv));
    }
    w[i] = a;
    Mw[i] = b;
  }
}

// In-place basis rotation V[:, 0:k] = V[:, 0:m] Y (Y real, m x k, column-major).
// Each block stages TE elements of all m vectors in shared memory first.
template <int TE>
__global__ void k_rotate_basis(double2* __restrict__ V, int m, const double* __restrict__ Y, int k, long long N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tile = reinterpret_cast<double2*>(smem_raw);  // [m][TE]
  for (long long base = (long long)blockIdx.x * TE; base < N; base += (long long)gridDim.x * TE) {
    for (int idx = threadIdx.x; idx < m * TE; idx += blockDim.x) {
      const int j = idx / TE, t = idx % TE;
      const long long i = base + t;
      tile[idx] = i < N ? V[(long long)j * N + i] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < k * TE; idx += blockDim.x) {
      const int col = idx / TE, t = idx % TE;
      const long long i = base + t;
      double2 acc = make_double2(0.0, 0.0);
      for (int j = 0; j < m; ++j) {
        const double y = Y[(long long)col * m + j];
        const double2 v = tile[j * TE + t];
        acc.x += y * v.x;
        acc.y += y * v.y;
      }
      if (i < N) V[(long long)col * N + i] = acc;
    }
    __syncthreads();
  }
}

}  // namespace nfs
