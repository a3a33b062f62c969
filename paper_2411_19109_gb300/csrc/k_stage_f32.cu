// Explicit instantiations of the RK4 stage row kernels in float (one translation unit per
// kernel family and precision so that nvcc compiles them in parallel).
#include "kernels_impl.cuh"

namespace llg {
template void launch_rows_mode<float, ROW_STAGE>(const RowArgs<float>&, int, size_t, cudaStream_t, bool);
template void smem_rows_mode<float, ROW_STAGE>(size_t);
}  // namespace llg
