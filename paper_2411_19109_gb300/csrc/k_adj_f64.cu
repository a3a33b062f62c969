// Explicit instantiations of the adjoint stage kernels in double (one translation unit per
// kernel family and precision so that nvcc compiles them in parallel).
#include "kernels_impl.cuh"

namespace llg {
template void launch_adj<double>(const AdjArgs<double>&, int, size_t, cudaStream_t, bool, int);
template void smem_adj<double>(size_t);
}  // namespace llg
