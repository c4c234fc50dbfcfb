// server.cu -- the serving kernel for contexts without pruned nodes, and the
// dispatch between the two serving kernels (server_nodes.cu holds the other).
#include <mutex>

#include "server_kernel.cuh"

namespace pscl {

cudaError_t srv_prepare_nodes(size_t smem, int *bps);
cudaError_t srv_launch_nodes(const SrvParams &S, int grid, size_t smem, cudaStream_t s);

static std::mutex g_srv_attr_mu;

cudaError_t server_attrs(bool nodes, size_t smem, int *bps)
{
    std::lock_guard<std::mutex> lk(g_srv_attr_mu);
    return nodes ? srv_prepare_nodes(smem, bps) : srv_prepare<false>(smem, bps);
}

cudaError_t server_launch(bool nodes, const SrvParams &S, int grid, size_t smem, cudaStream_t s)
{
    return nodes ? srv_launch_nodes(S, grid, smem, s) : srv_launch<false>(S, grid, smem, s);
}

}  // namespace pscl
