// The A_r product in double-single arithmetic (R = df, C = dfc: float pairs
// hi + lo, about 48 bits; see dfloat.cuh).  Used for the FP64-accuracy
// refinement residuals of the mixed-precision path, where it replaces the
// complex128 product: this GPU's FP32 units are far faster than its FP64 ones.
#include "dfloat.cuh"
#include "matvec_impl.cuh"

namespace nfs {

NFS_INSTANTIATE_MATVEC(df)

// complex128 <-> double-single conversions of `count` reals
__global__ void k_double_to_df(const double* __restrict__ in, df* __restrict__ out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = df(in[i]);
}
__global__ void k_df_to_double(const df* in, double* out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const df v = in[i];  // read before the write: in and out may be the same buffer
    out[i] = (double)v;
  }
}

cudaError_t double_to_df(const double* in, df* out, long long count, cudaStream_t s) {
  const int blocks = (int)std::min<long long>((count + 255) / 256, 152LL * 16);
  k_double_to_df<<<blocks, 256, 0, s>>>(in, out, count);
  return cudaGetLastError();
}
cudaError_t df_to_double(const df* in, double* out, long long count, cudaStream_t s) {
  const int blocks = (int)std::min<long long>((count + 255) / 256, 152LL * 16);
  k_df_to_double<<<blocks, 256, 0, s>>>(in, out, count);
  return cudaGetLastError();
}

}  // namespace nfs
