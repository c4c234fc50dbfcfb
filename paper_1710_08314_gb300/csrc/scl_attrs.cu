// scl_attrs.cu -- occupancy query dispatch over the number formats.
#include "internal.h"

namespace pscl {
cudaError_t scl_attrs_f32(int kv, size_t smem, int block, int *bps);
cudaError_t scl_attrs_i16(int kv, size_t smem, int block, int *bps);
cudaError_t scl_attrs_i8(int kv, size_t smem, int block, int *bps);

cudaError_t scl_func_attrs(int quant, int kv, size_t smem, int block, int *blocks_per_sm)
{
    if (quant == 0) return scl_attrs_f32(kv, smem, block, blocks_per_sm);
    if (quant == 1) return scl_attrs_i16(kv, smem, block, blocks_per_sm);
    return scl_attrs_i8(kv, smem, block, blocks_per_sm);
}
}  // namespace pscl
