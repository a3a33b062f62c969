// Explicit instantiation of the 16-element film column kernel in float (own
// translation unit so that it compiles in parallel with the others).
#include "cols16.cuh"

namespace llg {
template void launch_cols16<float>(const ColArgs<float>&, int, size_t, cudaStream_t);
template void smem_cols16<float>(size_t);
}  // namespace llg
