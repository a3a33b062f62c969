// Explicit instantiations of the spectrum / field / terminal row kernels in float (one translation unit per
// kernel family and precision so that nvcc compiles them in parallel).
#include "kernels_impl.cuh"

namespace llg {
template void launch_rows_mode<float, ROW_FFT_ONLY>(const RowArgs<float>&, int, size_t, cudaStream_t, bool);
template void launch_rows_mode<float, ROW_FIELD>(const RowArgs<float>&, int, size_t, cudaStream_t, bool);
template void launch_rows_mode<float, ROW_TERMINAL>(const RowArgs<float>&, int, size_t, cudaStream_t, bool);
template void smem_rows_mode<float, ROW_FFT_ONLY>(size_t);
template void smem_rows_mode<float, ROW_FIELD>(size_t);
template void smem_rows_mode<float, ROW_TERMINAL>(size_t);
}  // namespace llg
