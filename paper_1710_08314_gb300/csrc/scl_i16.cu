// scl_i16.cu -- the list kernel for the i16 number format without the pruned-node
// handlers: 5 blocks of 4 warps per SM (96 registers) or 7 (72 registers).
#include "scl_launch.cuh"

PSCL_SCL_UNIT(plain_i16, QI16, false, 5, 7)
