// scl_launch.cuh -- launchers of the list kernel's variants.  A translation
// unit includes this for one (number format, node handlers) pair and
// instantiates the kernel at two register caps: MINB_LO and MINB_HI blocks
// of 128 threads per SM (lower and higher occupancy).
#pragma once
#include <map>
#include <mutex>

#include "scl_kernel.cuh"

namespace pscl {

template <class Qt, bool NODES, int MINB_LO, int MINB_HI>
struct SclLaunch {
    // the opt-in shared-memory limit, once per device
    static cudaError_t ensure()
    {
        static std::mutex mu;
        static std::map<int, int> done;
        int dev;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lk(mu);
        if (done[dev]) return cudaSuccess;
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(scl_kernel<Qt, NODES, MINB_LO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(scl_kernel<Qt, NODES, MINB_HI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin);
        if (e == cudaSuccess) done[dev] = 1;
        return e;
    }
    static cudaError_t launch(const KParams &p, bool hi, int grid, int block, size_t smem, cudaStream_t s)
    {
        cudaError_t e = ensure();
        if (e != cudaSuccess) return e;
        if (hi) scl_kernel<Qt, NODES, MINB_HI><<<grid, block, smem, s>>>(p);
        else scl_kernel<Qt, NODES, MINB_LO><<<grid, block, smem, s>>>(p);
        return cudaGetLastError();
    }
    static cudaError_t attrs(bool hi, size_t smem, int block, int *bps)
    {
        cudaError_t e = ensure();
        if (e != cudaSuccess) return e;
        if (hi) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, scl_kernel<Qt, NODES, MINB_HI>, block, smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, scl_kernel<Qt, NODES, MINB_LO>, block, smem);
    }
};

}  // namespace pscl

// one translation unit's entry points: launch_scl_<NAME> and attrs_scl_<NAME>
#define PSCL_SCL_UNIT(NAME, QT, NODES, LO, HI)                                                          \
    namespace pscl {                                                                                   \
    cudaError_t launch_scl_##NAME(const KParams &p, bool hi, int grid, int block, size_t smem,        \
                                  cudaStream_t s)                                                      \
    {                                                                                                  \
        return SclLaunch<QT, NODES, LO, HI>::launch(p, hi, grid, block, smem, s);                     \
    }                                                                                                  \
    cudaError_t attrs_scl_##NAME(bool hi, size_t smem, int block, int *bps)                            \
    {                                                                                                  \
        return SclLaunch<QT, NODES, LO, HI>::attrs(hi, smem, block, bps);                              \
    }                                                                                                  \
    }
