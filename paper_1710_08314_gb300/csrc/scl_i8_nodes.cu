// scl_i8_nodes.cu -- the list kernel for the i8 number format with the
// pruned-node handlers: 4 blocks of 4 warps per SM (128 registers) or 7 (72).
#include "scl_launch.cuh"

PSCL_SCL_UNIT(nodes_i8, QI8, true, 4, 7)
