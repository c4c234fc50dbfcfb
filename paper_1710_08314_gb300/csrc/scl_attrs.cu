// scl_attrs.cu -- launch and occupancy dispatch of the list kernel over the
// number formats and variants.
#include "internal.h"

namespace pscl {
#define PSCL_DECL(NAME)                                                                                  \
    cudaError_t launch_scl_##NAME(const KParams &p, bool hi, int grid, int block, size_t smem, cudaStream_t s); \
    cudaError_t attrs_scl_##NAME(bool hi, size_t smem, int block, int *bps);
PSCL_DECL(plain_f32)
PSCL_DECL(plain_i16)
PSCL_DECL(plain_i8)
PSCL_DECL(nodes_f32)
PSCL_DECL(nodes_i16)
PSCL_DECL(nodes_i8)
#undef PSCL_DECL

static bool kv_nodes(int kv) { return kv == KV_NODES || kv == KV_NODES_DENSE; }
static bool kv_hi(int kv) { return kv == KV_DENSE || kv == KV_NODES_DENSE; }

cudaError_t launch_scl(int quant, int kv, const KParams &p, int grid, int block, size_t smem, cudaStream_t s)
{
    const bool hi = kv_hi(kv);
    if (kv_nodes(kv)) {
        if (quant == 0) return launch_scl_nodes_f32(p, hi, grid, block, smem, s);
        if (quant == 1) return launch_scl_nodes_i16(p, hi, grid, block, smem, s);
        return launch_scl_nodes_i8(p, hi, grid, block, smem, s);
    }
    if (quant == 0) return launch_scl_plain_f32(p, hi, grid, block, smem, s);
    if (quant == 1) return launch_scl_plain_i16(p, hi, grid, block, smem, s);
    return launch_scl_plain_i8(p, hi, grid, block, smem, s);
}

cudaError_t scl_func_attrs(int quant, int kv, size_t smem, int block, int *blocks_per_sm)
{
    const bool hi = kv_hi(kv);
    if (kv_nodes(kv)) {
        if (quant == 0) return attrs_scl_nodes_f32(hi, smem, block, blocks_per_sm);
        if (quant == 1) return attrs_scl_nodes_i16(hi, smem, block, blocks_per_sm);
        return attrs_scl_nodes_i8(hi, smem, block, blocks_per_sm);
    }
    if (quant == 0) return attrs_scl_plain_f32(hi, smem, block, blocks_per_sm);
    if (quant == 1) return attrs_scl_plain_i16(hi, smem, block, blocks_per_sm);
    return attrs_scl_plain_i8(hi, smem, block, blocks_per_sm);
}
}  // namespace pscl
