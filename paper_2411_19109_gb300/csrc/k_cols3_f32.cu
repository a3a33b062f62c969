// Explicit instantiation of the 3D column-pass kernel in float (its own
// translation unit: the kernel has one body per column length and padded z
// length).
#include "cols3.cuh"

namespace llg {
template void launch_cols3<float>(const ColArgs<float>&, int, size_t, cudaStream_t);
template void smem_cols3<float>(size_t);
}  // namespace llg
