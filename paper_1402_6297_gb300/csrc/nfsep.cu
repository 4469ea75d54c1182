// Kernels of the null space free standard problem for any nonsingular B
// (see nfsep.h).  The DFT passes are those of the A_r product
// (matvec_kernels.cuh); only the per-voxel step between the z transforms and
// the scalings around the product differ.
#include <algorithm>
#include <cmath>

#include "matvec_impl.cuh"
#include "nfsep.h"

namespace nfs {

namespace {

__device__ __forceinline__ double quarter_root_lq(const double2* lam, int n1, int n2, long long e) {
  const int i1 = (int)(e % n1);
  const int i2 = (int)((e / n1) % n2);
  const int i3 = (int)(e / ((long long)n1 * n2));
  const double lq = cabs2(lam[i1]) + cabs2(lam[n1 + i2]) + cabs2(lam[n1 + n2 + i3]);
  return sqrt(sqrt(lq));
}

__global__ void k_nfsep_prescale(const double2* __restrict__ y, double2* __restrict__ t,
                                 const double2* __restrict__ lam, int n1, int n2, long long n) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < 4 * n; g += (long long)gridDim.x * blockDim.x) {
    const long long e = g % n;
    t[g] = cscale(y[g], quarter_root_lq(lam, n1, n2, e));
  }
}

__global__ void k_nfsep_post(const double2* __restrict__ a, double2* __restrict__ out, const double2* __restrict__ lam,
                             int n1, int n2, long long n, const double2* __restrict__ v, double2 sigma) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < 4 * n; g += (long long)gridDim.x * blockDim.x) {
    const long long q = g / n, e = g % n;
    double2 r = cscale(a[((q + 2) & 3) * n + e], quarter_root_lq(lam, n1, n2, e));
    if (v != nullptr) r = csub(r, cmul(sigma, v[g]));
    out[g] = r;
  }
}

// (e_c, h_c) = B_c^{-1} (p_c, q_c) for the three components of one voxel
struct BinvVoxel {
  const double2* b;
  long long n, v;
  __device__ __forceinline__ void apply(int k, double2 p, double2 q, double scale, double2& e, double2& h) const {
    const double2* bk = b + (long long)(4 * k) * n + v;
    e = cscale(cadd(cmul(bk[0], p), cmul(bk[n], q)), scale);
    h = cscale(cadd(cmul(bk[2 * n], p), cmul(bk[3 * n], q)), scale);
  }
};

template <int N3, int TX, int NT>
__global__ void __launch_bounds__(NT)
k_pass2_z_nfsep(double2* __restrict__ fld, const double2* __restrict__ binv, const double2* __restrict__ twz, int ncols,
                double inv_n) {
  using C = double2;
  constexpr int LINES = 6 * TX;
  constexpr int PITCH = LINES + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* stw = buf + N3 * PITCH;
  for (int i = threadIdx.x; i < N3; i += NT) stw[i] = twz[i];
  const int col0 = blockIdx.x * TX;
  const long long n = (long long)ncols * N3;
  C* tile = fld + col0;
  // line l = f * TX + c: field f, column col0 + c
  auto gaddr = [&](int l, int z) { return tile + (long long)(l / TX) * n + (long long)z * ncols + (l % TX); };
  __syncthreads();  // twiddles
  smem_fft_io<true, N3, LINES, NT, 1, PITCH, true, false>(buf, stw, [&](int l, int z) { return ldg_c(gaddr(l, z)); },
                                                         NoPut{});
  for (int idx = threadIdx.x; idx < N3 * TX; idx += NT) {
    const int c = idx % TX, z = idx / TX;
    C* row = buf + z * PITCH + c;
    const BinvVoxel bv{binv, n, (long long)z * ncols + col0 + c};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      C e, h;
      bv.apply(k, row[k * TX], row[(3 + k) * TX], inv_n, e, h);
      row[k * TX] = h;        // projected by P_r^* in pass 3 (group 0)
      row[(3 + k) * TX] = e;  // projected by Q_r^* in pass 3 (group 1)
    }
  }
  __syncthreads();
  smem_fft_io<false, N3, LINES, NT, 1, PITCH, false, true>(buf, stw, NoGet{},
                                                          [&](int l, int z, C v) { *gaddr(l, z) = v; });
}

template <int N3, int TX, int NT>
__global__ void __launch_bounds__(NT)
k_fields_z_nfsep(const double2* __restrict__ fld, const double2* __restrict__ binv, const double2* __restrict__ twz,
                 int n1, int ncols, const double2* __restrict__ bloch, double inv_sqrt_n, double2* __restrict__ X) {
  using C = double2;
  constexpr int LINES = 6 * TX;
  constexpr int PITCH = LINES + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* stw = buf + N3 * PITCH;
  for (int i = threadIdx.x; i < N3; i += NT) stw[i] = twz[i];
  const int col0 = blockIdx.x * TX;
  const long long n = (long long)ncols * N3;
  const C* tile = fld + col0;
  auto gaddr = [&](int l, int z) { return tile + (long long)(l / TX) * n + (long long)z * ncols + (l % TX); };
  __syncthreads();
  smem_fft_io<true, N3, LINES, NT, 1, PITCH, true, false>(buf, stw, [&](int l, int z) { return ldg_c(gaddr(l, z)); },
                                                         NoPut{});
  const int n2 = ncols / n1;
  for (int idx = threadIdx.x; idx < N3 * TX; idx += NT) {
    const int c = idx % TX, z = idx / TX;
    const int col = col0 + c;
    const long long v = (long long)z * ncols + col;
    const C* row = buf + z * PITCH + c;
    const BinvVoxel bv{binv, n, v};
    const C d = cmul(cmul(bloch[col % n1], bloch[n1 + col / n1]), bloch[n1 + n2 + z]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      C e, h;
      bv.apply(k, row[k * TX], row[(3 + k) * TX], inv_sqrt_n, e, h);
      X[k * n + v] = cmul(d, e);
      X[(3 + k) * n + v] = cmul(d, h);
    }
  }
}

__global__ void k_zaxpy_basis(double2* __restrict__ w, const double2* __restrict__ V, long long N,
                              const double* __restrict__ c, int m, double sign) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* cs = reinterpret_cast<double2*>(smem_raw);
  for (int j = threadIdx.x; j < m; j += blockDim.x) cs[j] = make_double2(sign * c[2 * j], sign * c[2 * j + 1]);
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double2 a = w[i];
    for (int j = 0; j < m; ++j) a = csub(a, cmul(cs[j], V[(long long)j * N + i]));
    w[i] = a;
  }
}

__global__ void k_zscale_copy(const double2* __restrict__ src, double2* __restrict__ dst, double scale, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    dst[i] = cscale(src[i], scale);
}

// in place: a tile of TE elements of all m vectors in shared memory, then the
// k combinations written back
template <int TE>
__global__ void k_zrotate(double2* __restrict__ V, int m, const double* __restrict__ Y, int k, long long N) {
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
      const int o = idx / TE, t = idx % TE;
      const long long i = base + t;
      double2 acc = make_double2(0.0, 0.0);
      for (int r = 0; r < m; ++r) {
        const double2 y = make_double2(Y[2 * ((long long)r * k + o)], Y[2 * ((long long)r * k + o) + 1]);
        acc = cadd(acc, cmul(tile[r * TE + t], y));
      }
      if (i < N) V[(long long)o * N + i] = acc;
    }
    __syncthreads();
  }
}

// --- device-resident GMRES -------------------------------------------------

constexpr int kGsChunk = 512;   // elements of one dot-product chunk
constexpr int kGsMaxChunks = 64;
constexpr int kGsThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the block (blockDim.x = kGsThreads); the result in every thread
__device__ __forceinline__ double gs_block_sum(double v, double* red) {
  v = warp_sum(v);
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[wi] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < kGsThreads / 32; ++i) t += red[i];
  return t;
}

// grid (S, ceil(m / 8)): warp wi of block (s, b) forms chunk s of V_j^* w, j = 8 b + wi
__global__ void __launch_bounds__(kGsThreads)
k_gs_dots(const double2* __restrict__ V, int m, const double2* __restrict__ w, long long N, long long chunk,
          double* __restrict__ part) {
  const int j = blockIdx.y * (kGsThreads / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= m) return;  // whole warps
  const int s = blockIdx.x;
  const long long i0 = (long long)s * chunk, i1 = min(N, i0 + chunk);
  const double2* v = V + (long long)j * N;
  double re = 0.0, im = 0.0;
#pragma unroll 4
  for (long long i = i0 + lane; i < i1; i += 32) {
    const double2 a = v[i], b = w[i];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) {
    part[((long long)s * m + j) * 2] = re;
    part[((long long)s * m + j) * 2 + 1] = im;
  }
}

__global__ void __launch_bounds__(kGsThreads)
k_gs_axpy(double2* __restrict__ w, const double2* __restrict__ V, long long N, int m, const double* __restrict__ part,
          int S, double* __restrict__ nrm_part) {
  __shared__ double2 cs[kGmresMax];
  __shared__ double red[kGsThreads / 32];
  for (int j = threadIdx.x; j < m; j += kGsThreads) {
    double re = 0.0, im = 0.0;
    for (int q = 0; q < S; ++q) {
      re += part[((long long)q * m + j) * 2];
      im += part[((long long)q * m + j) * 2 + 1];
    }
    cs[j] = make_double2(re, im);
  }
  __syncthreads();
  double nr = 0.0;
  for (long long i = (long long)blockIdx.x * kGsThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kGsThreads) {
    // eight basis loads in flight per round, two accumulators
    double2 a0 = w[i], a1 = make_double2(0.0, 0.0);
    int j = 0;
    for (; j + 8 <= m; j += 8) {
      double2 v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = V[(long long)(j + t) * N + i];
#pragma unroll
      for (int t = 0; t < 8; t += 2) {
        a0 = csub(a0, cmul(cs[j + t], v[t]));
        a1 = csub(a1, cmul(cs[j + t + 1], v[t + 1]));
      }
    }
    for (; j < m; ++j) a0 = csub(a0, cmul(cs[j], V[(long long)j * N + i]));
    const double2 a = cadd(a0, a1);
    w[i] = a;
    nr += cabs2(a);
  }
  if (nrm_part) {
    nr = gs_block_sum(nr, red);
    if (threadIdx.x == 0) nrm_part[blockIdx.x] = nr;
  }
}

// Short vectors: grid (ceil(N / kGsThreads), chunks of kGsAxpyChunk basis
// vectors); tmp[jc N + i] = sum over chunk jc of c_j V_j[i]
constexpr int kGsAxpyChunk = 16;
__global__ void __launch_bounds__(kGsThreads)
k_gs_axpy_part(const double2* __restrict__ V, long long N, int m, const double* __restrict__ part, int S,
               double2* __restrict__ tmp) {
  __shared__ double2 cs[kGsAxpyChunk];
  const int j0 = blockIdx.y * kGsAxpyChunk;
  const int nj = min(kGsAxpyChunk, m - j0);
  if (threadIdx.x < nj) {
    double re = 0.0, im = 0.0;
    for (int q = 0; q < S; ++q) {
      re += part[((long long)q * m + j0 + threadIdx.x) * 2];
      im += part[((long long)q * m + j0 + threadIdx.x) * 2 + 1];
    }
    cs[threadIdx.x] = make_double2(re, im);
  }
  __syncthreads();
  const long long i = (long long)blockIdx.x * kGsThreads + threadIdx.x;
  if (i >= N) return;
  double2 v[kGsAxpyChunk];
#pragma unroll
  for (int t = 0; t < kGsAxpyChunk; ++t) v[t] = t < nj ? V[(long long)(j0 + t) * N + i] : make_double2(0.0, 0.0);
  double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
#pragma unroll
  for (int t = 0; t < kGsAxpyChunk; t += 2) {
    if (t < nj) a0 = cadd(a0, cmul(cs[t], v[t]));
    if (t + 1 < nj) a1 = cadd(a1, cmul(cs[t + 1], v[t + 1]));
  }
  tmp[(long long)blockIdx.y * N + i] = cadd(a0, a1);
}

// w -= sum over the JC partial sums in tmp, and the partials of ||w||^2
__global__ void __launch_bounds__(kGsThreads)
k_gs_axpy_sum(double2* __restrict__ w, long long N, const double2* __restrict__ tmp, int JC,
              double* __restrict__ nrm_part) {
  __shared__ double red[kGsThreads / 32];
  double nr = 0.0;
  for (long long i = (long long)blockIdx.x * kGsThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kGsThreads) {
    double2 a = w[i];
    for (int jc = 0; jc < JC; ++jc) a = csub(a, tmp[(long long)jc * N + i]);
    w[i] = a;
    nr += cabs2(a);
  }
  if (nrm_part) {
    nr = gs_block_sum(nr, red);
    if (threadIdx.x == 0) nrm_part[blockIdx.x] = nr;
  }
}

__global__ void __launch_bounds__(kGsThreads)
k_gmres_residual(const double2* __restrict__ b, double2* __restrict__ w, long long N, double* __restrict__ nrm_part) {
  __shared__ double red[kGsThreads / 32];
  double nr = 0.0;
  for (long long i = (long long)blockIdx.x * kGsThreads + threadIdx.x; i < N; i += (long long)gridDim.x * kGsThreads) {
    const double2 a = csub(b[i], w[i]);
    w[i] = a;
    nr += cabs2(a);
  }
  nr = gs_block_sum(nr, red);
  if (threadIdx.x == 0) nrm_part[blockIdx.x] = nr;
}

__device__ __forceinline__ double gs_sum_partials(const double* part, int nb, double* red) {
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += kGsThreads) t += part[b];
  return gs_block_sum(t, red);
}

__global__ void __launch_bounds__(kGsThreads)
k_gmres_column(int j, const double* __restrict__ part1, const double* __restrict__ part2, int S,
               const double* __restrict__ nrm_part, int nb, GmresDev* st) {
  __shared__ double red[kGsThreads / 32];
  if (st->done) {  // the same value in every thread: nothing below writes it before this point
    if (threadIdx.x == 0) st->inv_h = 0.0;
    return;
  }
  const int m = j + 1;  // vectors the two passes ran over
  double2* col = st->Hc + (long long)j * (kGmresMax + 1);
  for (int i = threadIdx.x; i < m; i += kGsThreads) {
    double re = 0.0, im = 0.0;
    for (int q = 0; q < S; ++q) {
      re += part1[((long long)q * m + i) * 2] + part2[((long long)q * m + i) * 2];
      im += part1[((long long)q * m + i) * 2 + 1] + part2[((long long)q * m + i) * 2 + 1];
    }
    col[i] = make_double2(re, im);
  }
  const double h = sqrt(fmax(gs_sum_partials(nrm_part, nb, red), 0.0));
  if (threadIdx.x == 0) {
    col[j + 1] = make_double2(h, 0.0);
    st->done = h == 0.0 ? 1 : 0;
    st->inv_h = h > 0.0 ? 1.0 / h : 0.0;
  }
}

__global__ void k_gmres_store(const double2* __restrict__ w, double2* __restrict__ dst, const GmresDev* st, long long N) {
  const double sc = st->inv_h;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    dst[i] = cscale(w[i], sc);
}

int blocks_for(long long work) { return (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, 152LL * 16)); }

template <int N3>
cudaError_t prep_n3() {
  constexpr int TX = z_tile(N3, 16);
  constexpr int NT = z_threads(N3, 16);
  cudaError_t e = cudaFuncSetAttribute(k_pass2_z_nfsep<N3, TX, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)z_smem<double, N3>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fields_z_nfsep<N3, TX, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)z_smem<double, N3>());
}

template <int N3>
cudaError_t pass2_n3(double2* fld, const double2* binv, const double2* tw3, int ncols, cudaStream_t s) {
  constexpr int TX = z_tile(N3, 16);
  constexpr int NT = z_threads(N3, 16);
  k_pass2_z_nfsep<N3, TX, NT><<<ncols / TX, NT, z_smem<double, N3>(), s>>>(fld, binv, tw3, ncols,
                                                                         1.0 / ((double)ncols * N3));
  return cudaGetLastError();
}

template <int N3>
cudaError_t fields_n3(const double2* fld, const double2* binv, const double2* tw3, const double2* bloch, int n1,
                      int ncols, double2* X, cudaStream_t s) {
  constexpr int TX = z_tile(N3, 16);
  constexpr int NT = z_threads(N3, 16);
  k_fields_z_nfsep<N3, TX, NT><<<ncols / TX, NT, z_smem<double, N3>(), s>>>(
      fld, binv, tw3, n1, ncols, bloch, 1.0 / std::sqrt((double)ncols * N3), X);
  return cudaGetLastError();
}

}  // namespace

cudaError_t nfsep_prescale(const double2* y, double2* t, const double2* lam, int n1, int n2, int n3,
                           cudaStream_t s) {
  const long long n = (long long)n1 * n2 * n3;
  k_nfsep_prescale<<<blocks_for(4 * n), 256, 0, s>>>(y, t, lam, n1, n2, n);
  return cudaGetLastError();
}

cudaError_t nfsep_post(const double2* a, double2* out, const double2* lam, int n1, int n2, int n3,
                       const double2* v, double2 sigma, cudaStream_t s) {
  const long long n = (long long)n1 * n2 * n3;
  k_nfsep_post<<<blocks_for(4 * n), 256, 0, s>>>(a, out, lam, n1, n2, n, v, sigma);
  return cudaGetLastError();
}

cudaError_t nfsep_prepare(int n3) {
  switch (n3) {
#define NFS_CASE(N) case N: return prep_n3<N>();
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t nfsep_pass2(double2* fld, const double2* binv, const double2* tw3, int n1, int n2, int n3,
                        cudaStream_t s) {
  switch (n3) {
#define NFS_CASE(N) case N: return pass2_n3<N>(fld, binv, tw3, n1 * n2, s);
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t nfsep_fields(const double2* fld, const double2* binv, const double2* tw3, const double2* bloch,
                         int n1, int n2, int n3, double2* X, cudaStream_t s) {
  switch (n3) {
#define NFS_CASE(N) case N: return fields_n3<N>(fld, binv, tw3, bloch, n1, n1 * n2, X, s);
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t zaxpy_basis(double2* w, const double2* V, long long N, const double* c, int m, double sign,
                        cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  k_zaxpy_basis<<<blocks_for(N), 256, (size_t)m * sizeof(double2), s>>>(w, V, N, c, m, sign);
  return cudaGetLastError();
}

cudaError_t zscale_copy(const double2* src, double2* dst, double scale, long long N, cudaStream_t s) {
  k_zscale_copy<<<blocks_for(N), 256, 0, s>>>(src, dst, scale, N);
  return cudaGetLastError();
}

cudaError_t zrotate(double2* V, int m, const double* Y, int k, long long N, cudaStream_t s) {
  constexpr int TE = 32;
  const size_t smem = (size_t)m * TE * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_zrotate<TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((N + TE - 1) / TE, 152LL * 8));
  k_zrotate<TE><<<blocks, 256, smem, s>>>(V, m, Y, k, N);
  return cudaGetLastError();
}

int gs_chunks(long long N) {
  return (int)std::min<long long>(kGsMaxChunks, std::max<long long>(1, (N + kGsChunk - 1) / kGsChunk));
}

int gs_norm_blocks(long long N) { return blocks_for(N); }

// vectors shorter than this split the basis sum of gs_axpy across blocks
constexpr long long kGsSplitN = 152LL * 2 * kGsThreads;

long long gs_axpy_tmp_len(long long N) {
  return N < kGsSplitN ? (long long)((kGmresMax + kGsAxpyChunk - 1) / kGsAxpyChunk) * N : 0;
}

cudaError_t gs_dots(const double2* V, int m, const double2* w, long long N, double* part, cudaStream_t s) {
  if (m <= 0 || m > kGmresMax) return cudaErrorInvalidValue;
  const int S = gs_chunks(N);
  const long long chunk = (N + S - 1) / S;
  const dim3 grid(S, (m + kGsThreads / 32 - 1) / (kGsThreads / 32));
  k_gs_dots<<<grid, kGsThreads, 0, s>>>(V, m, w, N, chunk, part);
  return cudaGetLastError();
}

cudaError_t gs_axpy(double2* w, const double2* V, long long N, int m, const double* part, double* nrm_part,
                    double2* tmp, cudaStream_t s) {
  if (m <= 0 || m > kGmresMax) return cudaErrorInvalidValue;
  if (N < kGsSplitN) {
    if (tmp == nullptr) return cudaErrorInvalidValue;
    const int JC = (m + kGsAxpyChunk - 1) / kGsAxpyChunk;
    k_gs_axpy_part<<<dim3((unsigned)((N + kGsThreads - 1) / kGsThreads), JC), kGsThreads, 0, s>>>(V, N, m, part,
                                                                                                gs_chunks(N), tmp);
    k_gs_axpy_sum<<<gs_norm_blocks(N), kGsThreads, 0, s>>>(w, N, tmp, JC, nrm_part);
  } else {
    k_gs_axpy<<<gs_norm_blocks(N), kGsThreads, 0, s>>>(w, V, N, m, part, gs_chunks(N), nrm_part);
  }
  return cudaGetLastError();
}

int gs_axpy_kernels(long long N) { return N < kGsSplitN ? 2 : 1; }

cudaError_t gmres_residual(const double2* b, double2* w, long long N, double* nrm_part, cudaStream_t s) {
  k_gmres_residual<<<gs_norm_blocks(N), kGsThreads, 0, s>>>(b, w, N, nrm_part);
  return cudaGetLastError();
}

cudaError_t gmres_column(int j, const double* part1, const double* part2, int S, const double* nrm_part, int nb,
                         GmresDev* st, cudaStream_t s) {
  if (j < 0 || j >= kGmresMax) return cudaErrorInvalidValue;
  k_gmres_column<<<1, kGsThreads, 0, s>>>(j, part1, part2, S, nrm_part, nb, st);
  return cudaGetLastError();
}

cudaError_t gmres_store(const double2* w, double2* dst, const GmresDev* st, long long N, cudaStream_t s) {
  k_gmres_store<<<blocks_for(N), 256, 0, s>>>(w, dst, st, N);
  return cudaGetLastError();
}

}  // namespace nfs

