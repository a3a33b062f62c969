// Explicit instantiations of the adjoint stage kernel with FP32 node arrays
// and a double-float frequency domain, and of the double-float row
// transforms of the split adjoint stage (own translation unit so that it
// compiles in parallel with the others).
#include "kernels_impl.cuh"

namespace llg {
template void launch_adj<float, dfloat>(const AdjArgs<float, dfloat>&, int, size_t, cudaStream_t, bool, int);
template void smem_adj<float, dfloat>(size_t);
template void launch_spec_rows<float, dfloat>(const SpecRowArgs<float, dfloat>&, int, int, size_t, cudaStream_t);
template void smem_spec_rows<float, dfloat>(size_t);
}  // namespace llg
