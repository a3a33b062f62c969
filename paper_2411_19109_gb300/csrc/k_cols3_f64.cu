// Explicit instantiation of the 3D column-pass kernel in double (its own
// translation unit: the kernel has one body per column length and padded z
// length).
#include "cols3.cuh"

namespace llg {
template void launch_cols3<double>(const ColArgs<double>&, int, size_t, cudaStream_t);
template void smem_cols3<double>(size_t);
}  // namespace llg
