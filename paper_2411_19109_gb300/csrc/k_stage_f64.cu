// Explicit instantiations of the RK4 stage row kernels in double (one translation unit per
// kernel family and precision so that nvcc compiles them in parallel).
#include "kernels_impl.cuh"

namespace llg {
template void launch_rows_mode<double, ROW_STAGE>(const RowArgs<double>&, int, size_t, cudaStream_t, bool);
template void smem_rows_mode<double, ROW_STAGE>(size_t);
}  // namespace llg
