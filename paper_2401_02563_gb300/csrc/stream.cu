// Stream-mode edge-map kernels (relax_mode 3) for 32 and 64 lanes, and their dispatch.
#include "stream_kernel.cuh"

namespace kairos {

template cudaError_t stream_launch_w<32>(const StreamArgs &, int, int, cudaStream_t);
template cudaError_t stream_launch_w<64>(const StreamArgs &, int, int, cudaStream_t);
template int stream_max_blocks_w<32>(int);
template int stream_max_blocks_w<64>(int);

cudaError_t stream_launch(const StreamArgs &a, int W, int lam_bits, int grid, cudaStream_t s) {
    if (W == 64) return stream_launch_w<64>(a, lam_bits, grid, s);
    if (W == 32) return stream_launch_w<32>(a, lam_bits, grid, s);
    return cudaErrorInvalidValue;
}

int stream_max_grid(int W, int lam_bits, int sm_count, int *blocks_per_sm_out) {
    int nb = 0;
    if (W == 64) nb = stream_max_blocks_w<64>(lam_bits);
    else if (W == 32) nb = stream_max_blocks_w<32>(lam_bits);
    if (blocks_per_sm_out) *blocks_per_sm_out = nb;
    return nb * sm_count;
}

}  // namespace kairos
