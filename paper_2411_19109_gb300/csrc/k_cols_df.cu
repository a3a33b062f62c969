// Explicit instantiation of the film column kernel for the double-float
// frequency domain of the adjoint (own translation unit so that it compiles
// in parallel with the others).
#include "kernels_impl.cuh"

namespace llg {
template void launch_cols<dfloat>(const ColArgs<dfloat>&, int, size_t, cudaStream_t, int);
template void smem_cols<dfloat>(size_t);
}  // namespace llg
