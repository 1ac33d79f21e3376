// FP32 row kernels of the mixed-precision inner solve, padded block width 8.
#define MBPCG_KP 8
#include "inst_f32.inc"
