// Edge-map kernels of lane width 32 (both edge-time widths, every relaxation mode).
#include "edgemap_kernel.cuh"

namespace kairos {
template cudaError_t edgemap_launch_w<32>(const EdgeMapArgs &, int, int, cudaStream_t);
template int edgemap_max_blocks_w<32>(int, int);
}  // namespace kairos
