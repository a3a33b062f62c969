// Explicit instantiations of the Dormand-Prince row and adjoint kernels in float (own
// translation unit so that nvcc compiles them in parallel with the RK4 kernels).
#include "kernels_impl.cuh"

namespace llg {
template void launch_rows_mode<float, ROW_DP_STAGE>(const RowArgs<float>&, int, size_t, cudaStream_t, bool);
template void launch_rows_mode<float, ROW_DP_START>(const RowArgs<float>&, int, size_t, cudaStream_t, bool);
template void smem_rows_mode<float, ROW_DP_STAGE>(size_t);
template void smem_rows_mode<float, ROW_DP_START>(size_t);
template void launch_adj_dp<float>(const AdjArgs<float>&, int, size_t, cudaStream_t, bool);
template void smem_adj_dp<float>(size_t);
template void launch_dp_gather<float>(const DevInst*, const RowTile*, int, const float*, long long, const long long*,
                                       float*, cudaStream_t);
template void launch_dp_push<float>(const DevInst*, const RowTile*, int, const float*, float*, long long, const long long*,
                                   float*, cudaStream_t);
}  // namespace llg
