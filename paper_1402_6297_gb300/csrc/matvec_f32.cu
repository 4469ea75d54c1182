// complex64 instantiation of the three-pass A_r product.
#include "matvec_impl.cuh"

namespace nfs {
NFS_INSTANTIATE_MATVEC(float)
}  // namespace nfs
