// scl_i8.cu -- the list kernel for the i8 number format without the pruned-node
// handlers: 5 blocks of 4 warps per SM (96 registers) or 7 (72 registers).
#include "scl_launch.cuh"

PSCL_SCL_UNIT(plain_i8, QI8, false, 5, 7)
