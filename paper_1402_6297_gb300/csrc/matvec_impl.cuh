// Size dispatch and launch of the three matvec passes (see matvec_kernels.cuh).
// Included by matvec_f32.cu and matvec_f64.cu, which instantiate it.
#pragma once
#include "matvec.h"
#include "matvec_kernels.cuh"
#include "matvec_pk.cuh"
#include "matvec_split.cuh"

namespace nfs {

// Threads per CTA of the xy-plane passes, per plane edge length.
__host__ __device__ constexpr int plane_threads(int N) {
  return N == 8 ? 64 : N == 12 ? 64 : N == 16 ? 64 : N == 24 ? 128 : N == 32 ? 256
       : N == 48 ? 384 : N == 64 ? 256 : N == 96 ? 384 : 512;
}
// xy columns per CTA of the z pass, per z length and element size.
#ifndef NFS_ZTILE_C64
#define NFS_ZTILE_C64 16
#endif
#ifndef NFS_ZTHREADS_C64
#define NFS_ZTHREADS_C64 384
#endif
__host__ __device__ constexpr int z_tile(int N3, int csize) {
  return (csize == 16 && N3 >= 96) ? 8 : ((csize == 8 && N3 >= 48 && N3 <= 96) ? NFS_ZTILE_C64 : 16);
}
__host__ __device__ constexpr int z_threads(int N3, int csize) {
  return N3 == 128 ? 512 : ((csize == 8 && N3 >= 48 && N3 <= 96) ? NFS_ZTHREADS_C64 : 384);
}
// Minimum resident CTAs per SM requested from the compiler (caps registers so
// that three CTAs share an SM and overlap one's memory phase with the others'
// shared-memory FFTs; 96^3 complex64 planes are 75 KB, three fit in 228 KB).
// Only for complex64 and 48 <= N <= 96, where the shared memory allows it.
#ifndef NFS_PLANE_MINB
#define NFS_PLANE_MINB 3
#endif
#ifndef NFS_Z_MINB
#define NFS_Z_MINB 3
#endif
__host__ __device__ constexpr int plane_minb(int N, int csize) {
  return (csize == 8 && N >= 48 && N <= 96) ? NFS_PLANE_MINB : 1;
}
__host__ __device__ constexpr int z_minb(int N3, int csize) { return (csize == 8 && N3 >= 48 && N3 <= 96) ? NFS_Z_MINB : 1; }

template <typename R, int NX>
constexpr size_t plane_smem() {
  return (size_t)(NX * (NX + 1) + 2 * NX) * sizeof(cplx<R>);
}
template <typename R, int N3>
constexpr size_t z_smem() {
  return (size_t)(N3 * (6 * z_tile(N3, (int)sizeof(cplx<R>)) + 1) + N3) * sizeof(cplx<R>);
}

template <typename R, int NX>
constexpr bool plane_fits() {
  return plane_smem<R, NX>() <= kMaxDynSmem;
}

// Planes that do not fit run the five-pass product (matvec_split.cuh):
// tiles of kSplitRows rows (all three components) and kSplitCols columns.
constexpr int kSplitRows = 32;
constexpr int kSplitCols = 16;
constexpr int kSplitRowThreads = 512;
constexpr int kSplitColThreads = 128;
template <typename R, int NX>
constexpr size_t split_row_smem() {
  return (size_t)(3 * kSplitRows * (NX + 1) + NX) * sizeof(cplx<R>);
}
template <typename R, int NY>
constexpr size_t split_col_smem() {
  return (size_t)(NY * (kSplitCols + 1) + NY) * sizeof(cplx<R>);
}
// NFS_SPLIT_C64 = 1 runs the complex64 product in the five-pass form wherever
// the tiles divide the plane (smaller CTAs, more warps per SM, two extra trips
// of the fields through L2); 0 keeps the cluster form wherever planes fit.
#ifndef NFS_SPLIT_C64
#define NFS_SPLIT_C64 0
#endif
template <typename R, int NX>
constexpr bool split_fits() {
  return (!plane_fits<R, NX>() || (NFS_SPLIT_C64 && sizeof(cplx<R>) == 8)) && NX % kSplitRows == 0 &&
         NX % kSplitCols == 0 && split_row_smem<R, NX>() <= kMaxDynSmem;
}

#define NFS_FOR_EACH_SIZE(M) M(8) M(12) M(16) M(24) M(32) M(48) M(64) M(96) M(128)

// The paired complex64 kernels (matvec_pk.cuh) replace the unpaired ones at
// the lengths they exist for; NFS_PK = 0 keeps the unpaired kernels everywhere.
#ifndef NFS_PK
#define NFS_PK 1
#endif
template <typename R, int N>
constexpr bool use_pk() {
  return NFS_PK && std::is_same<R, float>::value && pk_plane_used(N) && pk_plane_smem<N>() <= kMaxDynSmem;
}
// Pass 3 in the paired form (1) or the unpaired cluster form (0): the paired
// pass 3 needs its own projection kernel (a CTA holds one component of the
// pair), which costs more than it saves.
#ifndef NFS_PK3
#define NFS_PK3 0
#endif
template <typename R, int N>
constexpr bool use_pk3() {
  return NFS_PK3 && use_pk<R, N>();
}
template <typename R, int N3>
constexpr bool use_pk_z() {
  return NFS_PK && std::is_same<R, float>::value && pk_z_used(N3) && pk_z_smem<N3>() <= kMaxDynSmem;
}

template <typename R, int NX>
static cudaError_t plane_prepare() {
  if constexpr (use_pk<R, NX>()) {
    constexpr int NT1 = pk_plane_threads(NX, 1), MB1 = pk_plane_minb(NX, 1);
    constexpr int NT3 = pk_plane_threads(NX, 3), MB3 = pk_plane_minb(NX, 3);
    cudaError_t e = cudaFuncSetAttribute(k_pk_pass1<NX, NT1, MB1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pk_plane_smem<NX>());
    if (e != cudaSuccess) return e;
    if constexpr (use_pk3<R, NX>()) {
      return cudaFuncSetAttribute(k_pk_pass3<NX, NT3, MB3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pk_plane_smem<NX>());
    } else {
      constexpr int NT = plane_threads(NX);
      return cudaFuncSetAttribute(k_pass3_fft_xy_project<R, NX, NX, NT, plane_minb(NX, (int)sizeof(cplx<R>))>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem<R, NX>());
    }
  } else if constexpr (split_fits<R, NX>()) {
    cudaError_t e = cudaFuncSetAttribute(k_pass1a_assemble_fft_x<R, NX, kSplitRows, kSplitRowThreads>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_row_smem<R, NX>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_pass3b_fft_x_project<R, NX, kSplitRows, kSplitRowThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_row_smem<R, NX>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fft_y_columns<true, R, NX, kSplitCols, kSplitColThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_col_smem<R, NX>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fft_y_columns<false, R, NX, kSplitCols, kSplitColThreads>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_col_smem<R, NX>());
  } else if constexpr (plane_fits<R, NX>()) {
    constexpr int NT = plane_threads(NX);
    cudaError_t e = cudaFuncSetAttribute(k_pass1_assemble_ifft_xy<R, NX, NX, NT, plane_minb(NX, (int)sizeof(cplx<R>))>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem<R, NX>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_pass3_fft_xy_project<R, NX, NX, NT, plane_minb(NX, (int)sizeof(cplx<R>))>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem<R, NX>());
    return e;
  } else {
    return cudaErrorInvalidValue;
  }
}

template <typename R, int N3>
static cudaError_t z_prepare() {
  if constexpr (use_pk_z<R, N3>()) {
    return cudaFuncSetAttribute(k_pk_pass2<N3, pk_z_threads(N3), pk_z_minb(N3)>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk_z_smem<N3>());
  }
  constexpr int TX = z_tile(N3, (int)sizeof(cplx<R>));
  constexpr int NT = z_threads(N3, (int)sizeof(cplx<R>));
  return cudaFuncSetAttribute(k_pass2_z_material<R, N3, TX, NT, z_minb(N3, (int)sizeof(cplx<R>))>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)z_smem<R, N3>());
}

template <typename R, int NX>
static cudaError_t plane_launch(const MatvecArgs<R>& a, int which) {
  if constexpr (use_pk<R, NX>()) {
    constexpr int NT1 = pk_plane_threads(NX, 1), MB1 = pk_plane_minb(NX, 1);
    constexpr int NT3 = pk_plane_threads(NX, 3), MB3 = pk_plane_minb(NX, 3);
    const dim3 grid(3, a.n3 * (a.P > 0 ? a.P : 1));
    if (which == 1) {
      if (a.cg_r != nullptr && (a.p_out == nullptr || (const void*)a.p_out == (const void*)a.u))
        return cudaErrorInvalidValue;  // the direction update needs its own output buffer
      k_pk_pass1<NX, NT1, MB1><<<grid, NT1, pk_plane_smem<NX>(), a.stream>>>(
          a.u, a.fld, a.lam, a.tw1, a.tw2, a.n3, a.alpha, a.beta, a.skip, a.cg_r, a.cg_beta, a.p_out, a.bs);
    } else if constexpr (use_pk3<R, NX>()) {
      if (a.cg.st != nullptr) return cudaErrorInvalidValue;  // no fused CG step in this form
      k_pk_pass3<NX, NT3, MB3><<<grid, NT3, pk_plane_smem<NX>(), a.stream>>>(a.fld, a.tw1, a.tw2, a.n3, a.skip,
                                                                             a.bs);
      constexpr int per_plane = (NX * NX + kProjThreads * kProjV - 1) / (kProjThreads * kProjV);
      k_pk_project<NX><<<per_plane * a.n3 * (a.P > 0 ? a.P : 1), kProjThreads, 0, a.stream>>>(
          a.fld, a.Au, a.lam, a.n3, a.alpha, a.beta, a.skip, a.bs);
    } else {
      constexpr int NT = plane_threads(NX);
      dim3 grid3(3, 2, a.n3 * (a.P > 0 ? a.P : 1));
      k_pass3_fft_xy_project<R, NX, NX, NT, plane_minb(NX, (int)sizeof(cplx<R>))>
          <<<grid3, NT, plane_smem<R, NX>(), a.stream>>>(a.fld, a.Au, a.lam, a.tw1, a.tw2, a.n3, a.alpha, a.beta,
                                                          a.skip, a.basis, a.bs, a.cg);
    }
    return cudaGetLastError();
  } else if constexpr (split_fits<R, NX>()) {
    if (a.cg.st != nullptr) return cudaErrorInvalidValue;  // no fused CG step in the five-pass form
    const int P = a.P > 0 ? a.P : 1;
    const dim3 rows(a.n2 / kSplitRows, 2, a.n3 * P), cols(a.n1 / kSplitCols, 6, a.n3 * P);
    if (which == 1) {
      k_pass1a_assemble_fft_x<R, NX, kSplitRows, kSplitRowThreads>
          <<<rows, kSplitRowThreads, split_row_smem<R, NX>(), a.stream>>>(
              a.u, a.fld, a.lam, a.tw1, a.n2, a.n3, a.alpha, a.beta, a.skip, a.cg_r, a.cg_beta, a.basis, a.bs);
      k_fft_y_columns<true, R, NX, kSplitCols, kSplitColThreads>
          <<<cols, kSplitColThreads, split_col_smem<R, NX>(), a.stream>>>(a.fld, a.tw2, a.n1, a.n3, a.skip, a.bs);
    } else {
      k_fft_y_columns<false, R, NX, kSplitCols, kSplitColThreads>
          <<<cols, kSplitColThreads, split_col_smem<R, NX>(), a.stream>>>(a.fld, a.tw2, a.n1, a.n3, a.skip, a.bs);
      k_pass3b_fft_x_project<R, NX, kSplitRows, kSplitRowThreads>
          <<<rows, kSplitRowThreads, split_row_smem<R, NX>(), a.stream>>>(
              a.fld, a.Au, a.lam, a.tw1, a.n2, a.n3, a.alpha, a.beta, a.skip, a.u, a.dot_part, a.basis, a.bs);
    }
    return cudaGetLastError();
  } else if constexpr (plane_fits<R, NX>()) {
    constexpr int NT = plane_threads(NX);
    dim3 grid(3, 2, a.n3 * (a.P > 0 ? a.P : 1));
    if (which == 1) {
      k_pass1_assemble_ifft_xy<R, NX, NX, NT, plane_minb(NX, (int)sizeof(cplx<R>))><<<grid, NT, plane_smem<R, NX>(), a.stream>>>(
          a.u, a.fld, a.lam, a.tw1, a.tw2, a.n3, a.alpha, a.beta, a.skip, a.cg_r, a.cg_beta, a.basis, a.bs);
    } else {
      k_pass3_fft_xy_project<R, NX, NX, NT, plane_minb(NX, (int)sizeof(cplx<R>))><<<grid, NT, plane_smem<R, NX>(), a.stream>>>(
          a.fld, a.Au, a.lam, a.tw1, a.tw2, a.n3, a.alpha, a.beta, a.skip, a.basis, a.bs, a.cg);
    }
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;
  }
}

template <typename R>
static bool split_rt(int n);

template <typename R, int N3>
static cudaError_t z_launch(const MatvecArgs<R>& a) {
  if constexpr (use_pk_z<R, N3>()) {
    static_assert(kPkZTile == z_tile(N3, 8), "one CG curvature partial per CTA of either z pass");
    const int ncols = a.n1 * a.n2;
    MatView<float> mv{a.inv_phi, a.gam, a.inv_mu, a.kind, a.ax_a, a.ax_b, (long long)ncols * a.n3};
    const float inv_n = (float)(1.0 / ((double)ncols * (double)a.n3));
    k_pk_pass2<N3, pk_z_threads(N3), pk_z_minb(N3)>
        <<<(ncols / kPkZTile) * (a.P > 0 ? a.P : 1), pk_z_threads(N3), pk_z_smem<N3>(), a.stream>>>(
            a.fld, mv, a.tw3, ncols, inv_n, a.skip, split_rt<R>(a.n1) ? nullptr : a.dot_part, a.bs);
    return cudaGetLastError();
  }
  constexpr int TX = z_tile(N3, (int)sizeof(cplx<R>));
  constexpr int NT = z_threads(N3, (int)sizeof(cplx<R>));
  const int ncols = a.n1 * a.n2;
  MatView<R> mv{a.inv_phi, a.gam, a.inv_mu, a.kind, a.ax_a, a.ax_b, (long long)ncols * a.n3};
  const R inv_n = (R)(1.0 / ((double)ncols * (double)a.n3));
  k_pass2_z_material<R, N3, TX, NT, z_minb(N3, (int)sizeof(cplx<R>))>
      <<<(ncols / TX) * (a.P > 0 ? a.P : 1), NT, z_smem<R, N3>(), a.stream>>>(
          a.fld, mv, a.tw3, ncols, inv_n, a.skip, split_rt<R>(a.n1) ? nullptr : a.dot_part, a.bs);
  return cudaGetLastError();
}

static inline bool size_ok(int n) {
  switch (n) {
    case 8: case 12: case 16: case 24: case 32: case 48: case 64: case 96: case 128: return true;
    default: return false;
  }
}

template <typename R>
static bool plane_fits_rt(int n) {
  switch (n) {
#define NFS_CASE(N) case N: return plane_fits<R, N>() || split_fits<R, N>();
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
    default: return false;
  }
}

template <typename R>
static int z_tile_rt(int n3) { return z_tile(n3, (int)sizeof(cplx<R>)); }

template <typename R>
bool matvec_supported(int n1, int n2, int n3) {
  if (n1 != n2 || !size_ok(n1) || !size_ok(n3)) return false;
  if (!plane_fits_rt<R>(n1)) return false;
  if ((n1 * n2) % z_tile_rt<R>(n3) != 0) return false;
  return true;
}

template <typename R>
cudaError_t matvec_prepare(int n1, int n2, int n3) {
  if (!matvec_supported<R>(n1, n2, n3)) return cudaErrorInvalidValue;
  cudaError_t e = cudaErrorInvalidValue;
  switch (n1) {
#define NFS_CASE(N) case N: e = plane_prepare<R, N>(); break;
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  if (e != cudaSuccess) return e;
  switch (n3) {
#define NFS_CASE(N) case N: e = z_prepare<R, N>(); break;
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return e;
}

template <typename R>
static cudaError_t plane_dispatch(const MatvecArgs<R>& a, int which) {
  switch (a.n1) {
#define NFS_CASE(N) case N: return plane_launch<R, N>(a, which);
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

template <typename R>
static cudaError_t z_dispatch(const MatvecArgs<R>& a) {
  switch (a.n3) {
#define NFS_CASE(N) case N: return z_launch<R, N>(a);
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t matvec_launch(const MatvecArgs<R>& a) {
  cudaError_t e = plane_dispatch<R>(a, 1);
  if (e != cudaSuccess) return e;
  e = z_dispatch<R>(a);
  if (e != cudaSuccess) return e;
  return plane_dispatch<R>(a, 3);
}

template <typename R>
cudaError_t matvec_launch_mask(const MatvecArgs<R>& a, int mask) {
  cudaError_t e = cudaSuccess;
  if (mask & 1) e = plane_dispatch<R>(a, 1);
  if (e == cudaSuccess && (mask & 2)) e = z_dispatch<R>(a);
  if (e == cudaSuccess && (mask & 4)) e = plane_dispatch<R>(a, 3);
  return e;
}

template <typename R>
cudaError_t pass1_launch(const MatvecArgs<R>& a) {
  return plane_dispatch<R>(a, 1);
}

template <typename R>
static bool split_rt(int n) {
  switch (n) {
#define NFS_CASE(N) case N: return split_fits<R, N>();
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return false;
}

template <typename R>
int matvec_dot_partials(int n1, int n2, int n3) {
  return split_rt<R>(n1) ? (n2 / kSplitRows) * 2 * n3 : (n1 * n2) / z_tile(n3, (int)sizeof(cplx<R>));
}

template <typename R>
bool cg_needs_p_out(int n1) {
  switch (n1) {
#define NFS_CASE(N) case N: return use_pk<R, N>();
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return false;
}

// Kernels one plane pass (1 or 3) launches: 1 in the cluster form, 2 in the
// five-pass form.
template <typename R>
int plane_pass_kernels(int n1) {
  return split_rt<R>(n1) ? 2 : 1;
}

// Kernels of one whole product: 3 in the cluster form, 5 in the five-pass
// form, 4 in the paired form (pass 3 and its projection kernel).
template <typename R>
bool cg_fusable(int n1) {
  if (split_rt<R>(n1)) return false;
  switch (n1) {
#define NFS_CASE(N) case N: return !use_pk3<R, N>();
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return false;
}

template <typename R>
int product_kernels(int n1) {
  if (split_rt<R>(n1)) return 5;
  switch (n1) {
#define NFS_CASE(N) case N: return use_pk3<R, N>() ? 4 : 3;
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return 3;
}

#define NFS_INSTANTIATE_MATVEC(R)                                            \
  template bool matvec_supported<R>(int, int, int);                        \
  template cudaError_t matvec_prepare<R>(int, int, int);                   \
  template cudaError_t matvec_launch<R>(const MatvecArgs<R>&);             \
  template cudaError_t matvec_launch_mask<R>(const MatvecArgs<R>&, int);   \
  template cudaError_t pass1_launch<R>(const MatvecArgs<R>&);               \
  template int matvec_dot_partials<R>(int, int, int);                      \
  template int plane_pass_kernels<R>(int);                                 \
  template bool cg_needs_p_out<R>(int);                                    \
  template int product_kernels<R>(int);                                    \
  template bool cg_fusable<R>(int);

}  // namespace nfs
