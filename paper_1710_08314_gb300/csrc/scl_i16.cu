// scl_i16.cu -- instantiations of the SCL kernel for the i16 number format
// (with the pruned-node handlers, and without them for 5 or 7 blocks per SM).
#include <map>
#include <mutex>

#include "scl_kernel.cuh"

namespace pscl {

static std::mutex g_attr_mu_i16;
static std::map<int, int> g_attr_set_i16;

static cudaError_t ensure_attr_i16()
{
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu_i16);
    if (g_attr_set_i16[dev]) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(scl_kernel<QI16, false, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(scl_kernel<QI16, true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(scl_kernel<QI16, false, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) g_attr_set_i16[dev] = 1;
    return e;
}

cudaError_t launch_scl_i16(const KParams &p, int kv, int grid, int block, size_t smem, cudaStream_t s)
{
    cudaError_t e = ensure_attr_i16();
    if (e != cudaSuccess) return e;
    if (kv == KV_NODES) scl_kernel<QI16, true, 4><<<grid, block, smem, s>>>(p);
    else if (kv == KV_DENSE) scl_kernel<QI16, false, 7><<<grid, block, smem, s>>>(p);
    else scl_kernel<QI16, false, 5><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t scl_attrs_i16(int kv, size_t smem, int block, int *bps)
{
    cudaError_t e = ensure_attr_i16();
    if (e != cudaSuccess) return e;
    if (kv == KV_NODES) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, scl_kernel<QI16, true, 4>, block, smem);
    if (kv == KV_DENSE) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, scl_kernel<QI16, false, 7>, block, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, scl_kernel<QI16, false, 5>, block, smem);
}

}  // namespace pscl
