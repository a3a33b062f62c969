// Explicit instantiations of the column-pass and elementwise kernels in double (one translation unit per
// kernel family and precision so that nvcc compiles them in parallel).
#include "kernels_impl.cuh"

namespace llg {
template void launch_cols<double>(const ColArgs<double>&, int, size_t, cudaStream_t, int);
template void smem_cols<double>(size_t);
template void launch_material_tiles<double>(const DevInst*, const RowTile*, int, const double*, double*, double*, double*, double*,
                                         cudaStream_t);
template void launch_grad_finish_tiles<double>(const DevInst*, const RowTile*, int, const double*, const double*,
                                            const double*, const double*, double*, const double*, double*, cudaStream_t);
template void launch_levelset_tiles<double>(const DevInst*, const RowTile*, int, double*, const double*,
                                         const unsigned char*, double, unsigned int*, cudaStream_t);
}  // namespace llg
