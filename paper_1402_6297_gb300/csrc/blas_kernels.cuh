// Vector kernels of the CG and Lanczos loops (Section 4.2: CG on A_r u = b;
// invert Lanczos on (B_r, A_r)), batched over the P problems of one context:
// problem p's vectors sit at base + p * N (N = 4n), and the problem index comes
// from a grid dimension, so a launch serves every problem at once.
//
// Reductions are deterministic: a grid of blocks per problem fixed by the
// vector length and the problem count (at most kRedBlocks) writes one
// partial per block, and a one-block kernel sums the partials in a fixed
// order.  Every CG kernel reads its problem's device `done` flag first and
// returns at once when it is set, so launched iterations past convergence (or
// for problems already converged) cost only empty launches.
#pragma once
#include <cstdint>
#include <type_traits>

#include "cg_state.cuh"
#include "nfs_complex.cuh"

namespace nfs {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0 (and warp 0) only.
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

__device__ __forceinline__ double sum_partials(const double* part, int count = kRedBlocks) {
  // one block of kRedThreads threads sums `count` partials in fixed order
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += kRedThreads) v += part[i];
  return block_sum<kRedThreads>(v);
}

// part[p * pstride + b] = block b's share of Re(conj(x_p) y_p); grid (blocks, P).
// skip (optional): problem p is skipped when skip[p * sstride] is nonzero.
template <typename C>
__global__ void __launch_bounds__(kRedThreads)
k_dot_re(const C* __restrict__ x, const C* __restrict__ y, long long N, double* __restrict__ part, long long pstride,
         const int* __restrict__ skip, int sstride) {
  const int p = blockIdx.y;
  if (skip && skip[(long long)p * sstride]) return;
  x += (long long)p * N;
  y += (long long)p * N;
  Acc<C> acc;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kRedThreads) {
    const C a = x[i], b = y[i];
    acc.add(a.x * b.x + a.y * b.y);
  }
  const double s = block_sum<kRedThreads>(acc.total());
  if (threadIdx.x == 0) part[(long long)p * pstride + blockIdx.x] = s;
}

// Partials of |Ay - omega By|^2 and |y|^2 for one eigenpair (the residual
// of the HHPD-NFGEP, B_r y = omega^{-1} A_r y scaled by omega): block b writes
// part[2b], part[2b + 1]; grid kRedBlocks.
__global__ void __launch_bounds__(kRedThreads)
k_residual_parts(const double2* __restrict__ Ay, const double2* __restrict__ By, const double2* __restrict__ y,
                 double omega, long long N, double* __restrict__ part) {
  double rr = 0.0, yy = 0.0;
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kRedThreads) {
    const double2 a = Ay[i], b = By[i], v = y[i];
    const double dx = a.x - omega * b.x, dy = a.y - omega * b.y;
    rr += dx * dx + dy * dy;
    yy += v.x * v.x + v.y * v.y;
  }
  rr = block_sum<kRedThreads>(rr);
  yy = block_sum<kRedThreads>(yy);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rr;
    part[2 * blockIdx.x + 1] = yy;
  }
}

// CG start, one block per problem: rr = the sum of the nred partials in
// part_a; stop once r^* r <= tol2[p].
__global__ void __launch_bounds__(kRedThreads)
k_cg_init(CGState* st, const double* __restrict__ tol2, int maxit, int npart_a, int nred) {
  st += blockIdx.x;
  const double rr = sum_partials(st->part_a, nred);
  if (threadIdx.x == 0) {
    const double t2 = tol2[blockIdx.x];
    st->npart_a = npart_a;
    st->rr = rr;
    st->tol2 = t2;
    st->it = 0;
    st->maxit = maxit;
    st->status = 0;
    st->alpha = st->beta = 0.0;
    st->arrived = 0;
    st->done = (rr <= t2) ? 1 : 0;
    if (!(rr == rr)) { st->done = 1; st->status = -7; }
  }
}

// One CG step after the product, for every problem (grid (kUpdBlocks, P)):
// alpha = rr / p^*Ap (every block sums the npart_a partials of p^* A p in the
// same order, so all blocks agree; block 0 records it), x += alpha p,
// r -= alpha Ap, and block b's partial of the new r^* r.  The last block to
// finish (counted with an atomic, no waiting) sums the partials in fixed
// order and sets beta = rr_new / rr, the convergence flag and the iteration
// count for the next launch.  Vectors move in 16-byte loads.
template <typename C>
__global__ void __launch_bounds__(kUpdThreads)
k_cg_update_xr(C* __restrict__ x, C* __restrict__ r, const C* __restrict__ p, const C* __restrict__ Ap, long long N,
               CGState* st) {
  const int pb = blockIdx.y;
  st += pb;
  if (st->done) return;
  using V = typename std::conditional<sizeof(C) == 8, float4, double2>::type;
  constexpr int EPV = 16 / (int)sizeof(C);
  V* x4 = reinterpret_cast<V*>(x + (long long)pb * N);
  V* r4 = reinterpret_cast<V*>(r + (long long)pb * N);
  const V* p4 = reinterpret_cast<const V*>(p + (long long)pb * N);
  const V* a4 = reinterpret_cast<const V*>(Ap + (long long)pb * N);
  using R = typename RealOf<C>::type;
  __shared__ double s_alpha;
  __shared__ int s_ok, s_last;
  double pAp;
  {
    double v = 0.0;
    for (int i = threadIdx.x; i < st->npart_a; i += kUpdThreads) v += st->part_a[i];
    pAp = block_sum<kUpdThreads>(v);  // valid in thread 0
  }
  if (threadIdx.x == 0) {
    s_alpha = st->rr / pAp;
    s_ok = (pAp > 0.0) && (s_alpha == s_alpha);  // also catches NaN
    if (blockIdx.x == 0) {
      st->pAp = pAp;
      st->alpha = s_alpha;
      if (!s_ok) {
        st->status = -7;
        st->done = 1;
      }
    }
  }
  __syncthreads();
  if (!s_ok) return;  // breakdown: leave x, r untouched (uniform per block)
  const R al = (R)s_alpha;
  Acc<C> acc;
  const long long NV = N / EPV;
  for (long long i = (long long)blockIdx.x * kUpdThreads + threadIdx.x; i < NV;
       i += (long long)gridDim.x * kUpdThreads) {
    const V pi = p4[i], ai = a4[i];
    V xi = x4[i], ri = r4[i];
    if constexpr (EPV == 2) {
      xi.x += al * pi.x; xi.y += al * pi.y; xi.z += al * pi.z; xi.w += al * pi.w;
      ri.x -= al * ai.x; ri.y -= al * ai.y; ri.z -= al * ai.z; ri.w -= al * ai.w;
      acc.add(ri.x * ri.x + ri.y * ri.y + ri.z * ri.z + ri.w * ri.w);
    } else {
      xi.x += al * pi.x; xi.y += al * pi.y;
      ri.x -= al * ai.x; ri.y -= al * ai.y;
      acc.add(ri.x * ri.x + ri.y * ri.y);
    }
    x4[i] = xi;
    r4[i] = ri;
  }
  const double s = block_sum<kUpdThreads>(acc.total());
  if (threadIdx.x == 0) {
    st->part_b[blockIdx.x] = s;
    __threadfence();
    s_last = atomicAdd(&st->arrived, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  // the last block: new residual norm, convergence, beta
  __threadfence();
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kUpdThreads) v += ((volatile double*)st->part_b)[i];
  const double rr = block_sum<kUpdThreads>(v);
  if (threadIdx.x == 0) {
    st->arrived = 0;
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

// ---------------------------------------------------------------------------
// Elementwise helpers over all P problems (flat index i, problem i / N)
// ---------------------------------------------------------------------------

template <typename C>
__global__ void k_sub(const C* __restrict__ a, const C* __restrict__ b, C* __restrict__ y, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    y[i] = csub(a[i], b[i]);
}

// Refinement residual per problem p (skip64, skip32: the masks of the two
// products just launched): r_p = b_p - Ap64_p where the complex128 product ran
// (!skip64[p]), else r_p -= s_p Ap32_p where the complex64 product of the
// correction ran (!skip32[p]), else r_p is left.  Grid-stride over P x N.
__global__ void k_refine_residual(double2* __restrict__ r, const double2* __restrict__ b,
                                  const double2* __restrict__ Ap64, const float2* __restrict__ Ap32,
                                  const double* __restrict__ s, const int* __restrict__ skip64,
                                  const int* __restrict__ skip32, long long N, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / N;
    if (!skip64[p]) {
      r[i] = csub(b[i], Ap64[i]);
    } else if (!skip32[p]) {
      const float2 a = Ap32[i];
      const double f = s[p];
      double2 ri = r[i];
      ri.x -= f * (double)a.x;
      ri.y -= f * (double)a.y;
      r[i] = ri;
    }
  }
}

// complex64 <- complex128 * s[problem]
__global__ void k_demote(const double2* __restrict__ a, const double* __restrict__ s, float2* __restrict__ y,
                         long long N, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = a[i];
    const double f = s[i / N];
    y[i] = make_float2((float)(v.x * f), (float)(v.y * f));
  }
}

// x += s[problem] * complex128(d)
__global__ void k_axpy_promote(double2* __restrict__ x, const double* __restrict__ s, const float2* __restrict__ d,
                               long long N, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = d[i];
    const double f = s[i / N];
    double2 xi = x[i];
    xi.x += f * (double)v.x;
    xi.y += f * (double)v.y;
    x[i] = xi;
  }
}

// B_r v = i [Sigma^{-1} v2 ; -Sigma^{-1} v1], Sigma_r = diag(sqrt(Lq), sqrt(Lq))
// (eq. NFSEP_spd_1).  lam holds Lambda_1 | Lambda_2 | Lambda_3 per problem
// (stride n1 + n2 + n3); v and out hold P vectors of 4n.
__global__ void k_apply_Br(const double2* __restrict__ v, double2* __restrict__ out, const double2* __restrict__ lam,
                           int n1, int n2, int n3, int P, long long vstride = -1) {
  const long long n = (long long)n1 * n2 * n3;
  const int nl = n1 + n2 + n3;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n * P; g += (long long)gridDim.x * blockDim.x) {
    const long long p = g / n, e = g % n;
    const int i1 = (int)(e % n1);
    const int i2 = (int)((e / n1) % n2);
    const int i3 = (int)(e / ((long long)n1 * n2));
    const double2* L = lam + p * nl;
    const double lq = cabs2(L[i1]) + cabs2(L[n1 + i2]) + cabs2(L[n1 + n2 + i3]);
    const double is = 1.0 / sqrt(lq);
    const double2* vp = v + p * (vstride >= 0 ? vstride : 4 * n);  // problem p's input (e.g. a basis column)
    double2* op = out + p * 4 * n;
    const double2 v1a = vp[e], v1b = vp[n + e], v2a = vp[2 * n + e], v2b = vp[3 * n + e];
    op[e] = cmul_i(cscale(v2a, is));
    op[n + e] = cmul_i(cscale(v2b, is));
    op[2 * n + e] = cmul_mi(cscale(v1a, is));
    op[3 * n + e] = cmul_mi(cscale(v1b, is));
  }
}

// Counter-based uniform numbers in [-1, 1) (splitmix64 finaliser of the
// element index and seed): the Lanczos starting vectors.
__device__ __forceinline__ double u01_hash(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// Problem p's starting vector at v + p * vstride (N entries).
__global__ void k_random_fill(double2* __restrict__ v, long long N, long long vstride, int P, unsigned long long seed) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N * P; g += (long long)gridDim.x * blockDim.x) {
    const long long p = g / N, i = g % N;
    const unsigned long long k = (unsigned long long)i * 2ull + seed * 0x632BE59BD9B4E019ull;
    v[p * vstride + i] = make_double2(u01_hash(k), u01_hash(k + 1));
  }
}

// ---------------------------------------------------------------------------
// Lanczos.  Problem p's basis: vector j at V + p * vstride + j * N (complex128),
// its new vector w at w + p * N.  Coefficients per problem at c + p * m * 2.
// ---------------------------------------------------------------------------

// part[((p * gridDim.x + b) * m + j) * 2 + {0,1}] = block b's share of
// conj(V_pj)^T w_p, j < m; grid (blocks, P).
template <int NT>
__global__ void __launch_bounds__(NT)
k_multi_dot(const double2* __restrict__ V, long long vstride, int m, const double2* __restrict__ w, long long N,
            double* __restrict__ part, const int* __restrict__ active) {
  constexpr int EPT = 4;  // elements of w per thread and pass
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  V += (long long)p * vstride;
  w += (long long)p * N;
  double* pp = part + ((long long)p * gridDim.x + blockIdx.x) * m * 2;
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
      pp[j0 * 2 + 0] = re;
      pp[j0 * 2 + 1] = im;
    }
  }
}

// out[(p * m + j) * 2 + {0,1}] = sum over nb blocks; grid (m, P)
__global__ void __launch_bounds__(kRedThreads)
k_multi_dot_finish(const double* __restrict__ part, int m, int nb, double* __restrict__ out,
                   const int* __restrict__ active) {
  const int j = blockIdx.x, p = blockIdx.y;
  if (active && !active[p]) return;
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nb; b += kRedThreads) {
    re += part[(((long long)p * nb + b) * m + j) * 2 + 0];
    im += part[(((long long)p * nb + b) * m + j) * 2 + 1];
  }
  re = block_sum<kRedThreads>(re);
  im = block_sum<kRedThreads>(im);
  if (threadIdx.x == 0) {
    out[((long long)p * m + j) * 2] = re;
    out[((long long)p * m + j) * 2 + 1] = im;
  }
}

// w_p -= sum_j c_pj V_pj ; Mw_p -= sum_j c_pj MV_pj; grid (blocks, P).
__global__ void k_multi_axpy(double2* __restrict__ w, double2* __restrict__ Mw, const double2* __restrict__ V,
                             const double2* __restrict__ MV, long long vstride, const double* __restrict__ c, int m,
                             long long N, const int* __restrict__ active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  w += (long long)p * N;
  Mw += (long long)p * N;
  V += (long long)p * vstride;
  MV += (long long)p * vstride;
  c += (long long)p * m * 2;
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

// Re-orthogonalisation through the shadows: w_p -= sum_j d_pj V32_pj and
// Mw_p -= sum_j d_pj MV32_pj for j < m, with d (layout of k_dots_finish, on the
// device) exact A_r inner products.  It runs only when the loss of
// orthogonality is small (|d| ~ 1e-8 of |w|), so the update is formed in FP32
// arithmetic from the FP32 shadows: its error is ~1e-8 * 6e-8 of |w|.
// Grid (blocks, P); problems with a zero flag are skipped.
__global__ void k_shadow_axpy(double2* __restrict__ w, double2* __restrict__ Mw, const float2* __restrict__ V32,
                              const float2* __restrict__ MV32, long long vstride, const double* __restrict__ d, int m,
                              long long N, const int* __restrict__ active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  w += (long long)p * N;
  Mw += (long long)p * N;
  V32 += (long long)p * vstride;
  MV32 += (long long)p * vstride;
  d += (long long)p * m * 2;
  // the coefficients as floats, converted once per block (double-precision
  // conversions run at the FP64 rate)
  extern __shared__ float2 sd[];
  for (int j = threadIdx.x; j < m; j += blockDim.x) sd[j] = make_float2((float)d[2 * j], (float)d[2 * j + 1]);
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      const float2 cj = sd[j];
      const float2 v = V32[(long long)j * N + i], mv = MV32[(long long)j * N + i];
      a = cadd(a, cmul(cj, v));
      b = cadd(b, cmul(cj, mv));
    }
    double2 wi = w[i], mi = Mw[i];
    wi.x -= (double)a.x;
    wi.y -= (double)a.y;
    mi.x -= (double)b.x;
    mi.y -= (double)b.y;
    w[i] = wi;
    Mw[i] = mi;
  }
}

// ---------------------------------------------------------------------------
// Exact A_r inner products on the FP32 units.  A_r is ill-conditioned
// (|A v| |w| >> |v|_A |w|_A), so single-precision inner products carry an
// absolute error near 1e-8 |w|_A: the level of orthogonality Lanczos needs to
// keep.  Here every operand is split into two floats (hi + lo, the lo part
// holding the FP64 remainder), the hi x hi products are formed exactly
// (TwoProduct by FMA) and summed exactly (TwoSum, Knuth), the small hi x lo
// and lo x hi terms and the rounding errors go to an ordinary FP32 sum, and
// the block sums are FP64: about 1e-14 of sum |terms|.  Double-precision
// arithmetic, scarce on this GPU, is used only for the per-block totals.
// ---------------------------------------------------------------------------

// Error-free transformations (TwoProduct by FMA; TwoSum, Knuth) on (real,
// imaginary) pairs, both halves in one packed f32x2 instruction:
// p + e = a * b and s + e = a + b exactly, per half.
__device__ __forceinline__ void two_prod_x2(float2 a, float2 b, float2& p, float2& e) {
  p = mul_x2(a, b);
  e = fma_x2(a, b, make_float2(-p.x, -p.y));
}
__device__ __forceinline__ void two_sum_x2(float2 a, float2 b, float2& s, float2& e) {
  s = add_x2(a, b);
  const float2 bb = sub_x2(s, a);
  e = add_x2(sub_x2(a, sub_x2(s, bb)), sub_x2(b, bb));
}
struct DSAccX2 {
  float2 hi = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
  __device__ __forceinline__ void add(float2 x) {
    float2 e;
    two_sum_x2(hi, x, hi, e);
    lo = add_x2(lo, e);
  }
};

__device__ __forceinline__ float2 split_lo(double2 v, float2 hi) {
  return make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
}

// In-place basis rotation V_p[:, 0:k] = V_p[:, 0:m] Y_p (Y_p real, m x k,
// column-major), in double-single arithmetic on the FP32 units: Y is given
// as float pairs Yhl[p m k + col m + j] = (hi, lo) with hi + lo = Y to ~1e-15,
// each block stages TE elements of all m vectors in shared memory split the
// same way, and every product hi x hi is formed exactly (TwoProduct) and
// summed exactly (TwoSum) with the cross terms and rounding errors in an
// ordinary FP32 sum: ~1e-14 of sum |terms|, at a small fraction of the cost
// of FP64 arithmetic (m k FP64 FMAs per element otherwise).  A thread forms
// CPT columns of one element.  Grid (blocks, P); problems with a zero flag
// are skipped.
template <int TE, int CPT>
__global__ void __launch_bounds__(256)
k_rotate_basis(double2* __restrict__ V, long long vstride, int m, const float2* __restrict__ Yhl, int k, long long N,
               const int* __restrict__ active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  V += (long long)p * vstride;
  Yhl += (long long)p * m * k;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* tile = reinterpret_cast<float4*>(smem_raw);  // [m][TE]: (re hi, im hi, re lo, im lo)
  const int groups = (k + CPT - 1) / CPT;
  for (long long base = (long long)blockIdx.x * TE; base < N; base += (long long)gridDim.x * TE) {
    for (int idx = threadIdx.x; idx < m * TE; idx += blockDim.x) {
      const int j = idx / TE, t = idx % TE;
      const long long i = base + t;
      const double2 v = i < N ? V[(long long)j * N + i] : make_double2(0.0, 0.0);
      const float2 h = make_float2((float)v.x, (float)v.y);
      const float2 l = split_lo(v, h);
      tile[idx] = make_float4(h.x, h.y, l.x, l.y);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < groups * TE; idx += blockDim.x) {
      const int g = idx / TE, t = idx % TE;
      const long long i = base + t;
      DSAccX2 acc[CPT];
      float2 small[CPT];
      const float2* yc[CPT];
#pragma unroll
      for (int q = 0; q < CPT; ++q) {
        small[q] = make_float2(0.f, 0.f);
        yc[q] = Yhl + (long long)min(g * CPT + q, k - 1) * m;  // columns past k: computed, not stored
      }
      for (int j = 0; j < m; ++j) {
        const float4 v = tile[j * TE + t];
        const float2 vh = make_float2(v.x, v.y), vl = make_float2(v.z, v.w);
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const float2 y = __ldg(yc[q] + j);
          const float2 yh = make_float2(y.x, y.x), yl = make_float2(y.y, y.y);
          float2 pr, e;
          two_prod_x2(yh, vh, pr, e);
          acc[q].add(pr);
          small[q] = add_x2(small[q], fma_x2(yh, vl, fma_x2(yl, vh, e)));
        }
      }
      if (i < N) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const int col = g * CPT + q;
          if (col < k)
            V[(long long)col * N + i] =
                make_double2((double)acc[q].hi.x + ((double)acc[q].lo.x + (double)small[q].x),
                             (double)acc[q].hi.y + ((double)acc[q].lo.y + (double)small[q].y));
        }
      }
    }
    __syncthreads();
  }
}

// out[(p * m + j) * 2 + {0,1}] = sum over the nb block partials of k_exact_dots; grid (m, P)
__global__ void __launch_bounds__(kRedThreads)
k_dots_finish(const double* __restrict__ part, int m, int nb, double* __restrict__ out, const int* __restrict__ active) {
  const int j = blockIdx.x, p = blockIdx.y;
  if (active && !active[p]) return;
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nb; b += kRedThreads) {
    re += part[(((long long)p * m + j) * nb + b) * 2 + 0];
    im += part[(((long long)p * m + j) * nb + b) * 2 + 1];
  }
  re = block_sum<kRedThreads>(re);
  im = block_sum<kRedThreads>(im);
  if (threadIdx.x == 0) {
    out[((long long)p * m + j) * 2] = re;
    out[((long long)p * m + j) * 2 + 1] = im;
  }
}

// part[(((p * m + j) * gridDim.x) + b) * 2 + {0, 1}] = block b's share of
// conj(S_pj)^T w_p (S = Shi + Slo, w = whi + wlo) for the G vectors
// j = blockIdx.y * G + g < m; grid (blocks, ceil(m / G), P).
template <int G>
__global__ void __launch_bounds__(kRedThreads)
k_exact_dots(const float2* __restrict__ Shi, const float2* __restrict__ Slo, long long sstride, int m,
             const float2* __restrict__ whi, const float2* __restrict__ wlo, long long N, double* __restrict__ part,
             const int* __restrict__ active) {
  const int p = blockIdx.z;
  if (active && !active[p]) return;
  Shi += (long long)p * sstride;
  Slo += (long long)p * sstride;
  whi += (long long)p * N;
  wlo += (long long)p * N;
  const int j0 = blockIdx.y * G;
  // per vector: the exact sum of the hi x hi products (real, imaginary) and
  // an ordinary sum of their rounding errors and the hi x lo, lo x hi terms
  DSAccX2 acc[G];
  float2 small[G];
#pragma unroll
  for (int g = 0; g < G; ++g) small[g] = make_float2(0.f, 0.f);
  for (long long i = (long long)blockIdx.x * kRedThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kRedThreads) {
    const float2 bh = whi[i], bl = wlo[i];
    // conj(a) b = (ar br + ai bi, ar bi - ai br) = ar (br, bi) + ai (bi, -br)
    const float2 bh2 = make_float2(bh.y, -bh.x), bl2 = make_float2(bl.y, -bl.x);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (j0 + g < m) {
        const float2 ah = Shi[(long long)(j0 + g) * N + i], al = Slo[(long long)(j0 + g) * N + i];
        const float2 ax = make_float2(ah.x, ah.x), ay = make_float2(ah.y, ah.y);
        float2 p1, e1, p2, e2;
        two_prod_x2(ax, bh, p1, e1);
        two_prod_x2(ay, bh2, p2, e2);
        acc[g].add(p1);
        acc[g].add(p2);
        float2 t = add_x2(e1, e2);
        t = fma_x2(ax, bl, t);
        t = fma_x2(make_float2(al.x, al.x), bh, t);
        t = fma_x2(ay, bl2, t);
        t = fma_x2(make_float2(al.y, al.y), bh2, t);
        small[g] = add_x2(small[g], t);
      }
    }
  }
  // block sums in FP64.  (Double-single sums on the FP32 units would free
  // the FP64 pipe, which these sums keep ~70% busy at small sizes, but they
  // lost the accuracy the monitor needs on homogeneous media at symmetric
  // k-points: spurious losses of 1e-6 and wrong degenerate eigenvalues.)
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const double sr = block_sum<kRedThreads>((double)acc[g].hi.x + (double)acc[g].lo.x + (double)small[g].x);
    const double si = block_sum<kRedThreads>((double)acc[g].hi.y + (double)acc[g].lo.y + (double)small[g].y);
    if (threadIdx.x == 0 && j0 + g < m) {
      const long long o = (((long long)p * m + j0 + g) * gridDim.x + blockIdx.x) * 2;
      part[o] = sr;
      part[o + 1] = si;
    }
  }
}

// w -> (whi, wlo) floats with whi + wlo = w to ~1e-15 (once per vector, so
// that the inner-product kernel runs no double-precision arithmetic)
__global__ void k_split_hi_lo(const double2* __restrict__ w, float2* __restrict__ whi, float2* __restrict__ wlo,
                              long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = w[i];
    const float2 h = make_float2((float)v.x, (float)v.y);
    whi[i] = h;
    wlo[i] = split_lo(v, h);
  }
}

// New basis vector j of every active problem: V_pj = s_p w_p, MV_pj = s_p Mw_p
// in FP64, plus their complex64 shadows and the FP64 remainder of the MV
// shadow (MV = MV32 + MV32lo to ~1e-15).
__global__ void k_store_basis_vector(const double2* __restrict__ w, const double2* __restrict__ Mw,
                                     const double* __restrict__ s, double2* __restrict__ V, double2* __restrict__ MV,
                                     float2* __restrict__ V32, float2* __restrict__ MV32, float2* __restrict__ MV32lo,
                                     long long vstride, int j, long long N, int P, const int* __restrict__ active) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N * P; g += (long long)gridDim.x * blockDim.x) {
    const long long p = g / N, i = g % N;
    if (active && !active[p]) continue;
    const double f = s[p];
    const double2 a = cscale(w[g], f), b = cscale(Mw[g], f);
    const long long o = p * vstride + (long long)j * N + i;
    V[o] = a;
    MV[o] = b;
    V32[o] = make_float2((float)a.x, (float)a.y);
    const float2 bh = make_float2((float)b.x, (float)b.y);
    MV32[o] = bh;
    MV32lo[o] = split_lo(b, bh);
  }
}

// Shadows of vectors [first, first + count) of every problem (after a basis
// rotation): V32, MV32 and MV32lo from V and MV.
__global__ void k_refresh_shadows(const double2* __restrict__ V, const double2* __restrict__ MV,
                                  float2* __restrict__ V32, float2* __restrict__ MV32, float2* __restrict__ MV32lo,
                                  long long vstride, long long len, int P) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < len * P; g += (long long)gridDim.x * blockDim.x) {
    const long long p = g / len, i = g % len;
    const long long o = p * vstride + i;
    const double2 a = V[o], b = MV[o];
    V32[o] = make_float2((float)a.x, (float)a.y);
    const float2 bh = make_float2((float)b.x, (float)b.y);
    MV32[o] = bh;
    MV32lo[o] = split_lo(b, bh);
  }
}

}  // namespace nfs
