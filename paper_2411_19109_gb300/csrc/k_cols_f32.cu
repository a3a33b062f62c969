// Explicit instantiations of the column-pass and elementwise kernels in float (one translation unit per
// kernel family and precision so that nvcc compiles them in parallel).
#include "kernels_impl.cuh"

namespace llg {
template void launch_cols<float>(const ColArgs<float>&, int, size_t, cudaStream_t, int);
template void smem_cols<float>(size_t);
template void launch_material_tiles<float>(const DevInst*, const RowTile*, int, const float*, float*, float*, double*, double*,
                                         cudaStream_t);
template void launch_grad_finish_tiles<float>(const DevInst*, const RowTile*, int, const float*, const float*,
                                            const float*, const double*, float*, const float*, float*, cudaStream_t);
template void launch_levelset_tiles<float>(const DevInst*, const RowTile*, int, float*, const float*,
                                         const unsigned char*, double, unsigned int*, cudaStream_t);
}  // namespace llg
