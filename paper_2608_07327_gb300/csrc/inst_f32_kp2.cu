// FP32 row kernels of the mixed-precision inner solve, padded block width 2.
#define MBPCG_KP 2
#include "inst_f32.inc"
