// FP32 row kernels of the mixed-precision inner solve, padded block width 1.
#define MBPCG_KP 1
#include "inst_f32.inc"
