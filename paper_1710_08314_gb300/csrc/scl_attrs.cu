// scl_attrs.cu -- occupancy query dispatch over the number formats.
#include "internal.h"

namespace pscl {
cudaError_t scl_attrs_f32(size_t smem, int block, int *bps);
cudaError_t scl_attrs_i16(size_t smem, int block, int *bps);
cudaError_t scl_attrs_i8(size_t smem, int block, int *bps);

cudaError_t scl_func_attrs(int quant, size_t smem, int block, int *blocks_per_sm)
{
    if (quant == 0) return scl_attrs_f32(smem, block, blocks_per_sm);
    if (quant == 1) return scl_attrs_i16(smem, block, blocks_per_sm);
    return scl_attrs_i8(smem, block, blocks_per_sm);
}
}  // namespace pscl
