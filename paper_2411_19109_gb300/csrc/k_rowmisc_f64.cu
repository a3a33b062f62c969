// Explicit instantiations of the spectrum / field / terminal row kernels in double (one translation unit per
// kernel family and precision so that nvcc compiles them in parallel).
#include "kernels_impl.cuh"

namespace llg {
template void launch_rows_mode<double, ROW_FFT_ONLY>(const RowArgs<double>&, int, size_t, cudaStream_t, bool);
template void launch_rows_mode<double, ROW_FIELD>(const RowArgs<double>&, int, size_t, cudaStream_t, bool);
template void launch_rows_mode<double, ROW_TERMINAL>(const RowArgs<double>&, int, size_t, cudaStream_t, bool);
template void smem_rows_mode<double, ROW_FFT_ONLY>(size_t);
template void smem_rows_mode<double, ROW_FIELD>(size_t);
template void smem_rows_mode<double, ROW_TERMINAL>(size_t);
}  // namespace llg
