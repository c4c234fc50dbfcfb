// server_nodes.cu -- the serving kernel for contexts with pruned nodes (its
// own translation unit so that the two serving kernels compile in parallel).
#include "server_kernel.cuh"

namespace pscl {

cudaError_t srv_prepare_nodes(size_t smem, int *bps) { return srv_prepare<true>(smem, bps); }

cudaError_t srv_launch_nodes(const SrvParams &S, int grid, size_t smem, cudaStream_t s)
{
    return srv_launch<true>(S, grid, smem, s);
}

}  // namespace pscl
