// Edge-map kernels of lane width 1 (both edge-time widths, every relaxation mode).
#include "edgemap_kernel.cuh"

namespace kairos {
template cudaError_t edgemap_launch_w<1>(const EdgeMapArgs &, int, int, cudaStream_t);
template int edgemap_max_blocks_w<1>(int, int);
}  // namespace kairos
