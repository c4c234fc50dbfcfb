// scl_i16_nodes.cu -- the list kernel for the i16 number format with the
// pruned-node handlers: 4 blocks of 4 warps per SM (128 registers) or 7 (72).
#include "scl_launch.cuh"

PSCL_SCL_UNIT(nodes_i16, QI16, true, 4, 7)
