// Explicit instantiations of the adjoint stage kernels in float (one translation unit per
// kernel family and precision so that nvcc compiles them in parallel).
#include "kernels_impl.cuh"

namespace llg {
template void launch_adj<float>(const AdjArgs<float>&, int, size_t, cudaStream_t, bool, int);
template void smem_adj<float>(size_t);
template void launch_adj_split<float>(const AdjArgs<float>&, int, size_t, cudaStream_t, int);
template void smem_adj_split<float>(size_t);
}  // namespace llg
