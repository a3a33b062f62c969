// Explicit instantiations of the Dormand-Prince row and adjoint kernels in double (own
// translation unit so that nvcc compiles them in parallel with the RK4 kernels).
#include "kernels_impl.cuh"

namespace llg {
template void launch_rows_mode<double, ROW_DP_STAGE>(const RowArgs<double>&, int, size_t, cudaStream_t, bool);
template void launch_rows_mode<double, ROW_DP_START>(const RowArgs<double>&, int, size_t, cudaStream_t, bool);
template void smem_rows_mode<double, ROW_DP_STAGE>(size_t);
template void smem_rows_mode<double, ROW_DP_START>(size_t);
template void launch_adj_dp<double>(const AdjArgs<double>&, int, size_t, cudaStream_t, bool);
template void smem_adj_dp<double>(size_t);
template void launch_dp_gather<double>(const DevInst*, const RowTile*, int, const double*, long long, const long long*,
                                       double*, cudaStream_t);
template void launch_dp_push<double>(const DevInst*, const RowTile*, int, const double*, double*, long long, const long long*,
                                   double*, cudaStream_t);
}  // namespace llg
