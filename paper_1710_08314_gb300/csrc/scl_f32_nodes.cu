// scl_f32_nodes.cu -- the list kernel for the f32 number format with the
// pruned-node handlers: 4 blocks of 4 warps per SM (128 registers) or 7 (72).
#include "scl_launch.cuh"

PSCL_SCL_UNIT(nodes_f32, QF32, true, 4, 7)
