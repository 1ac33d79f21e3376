// FP32 row kernels of the mixed-precision inner solve, padded block width 4.
#define MBPCG_KP 4
#include "inst_f32.inc"
