// FP32 row kernels of the mixed-precision inner solve, padded block width 16.
#define MBPCG_KP 16
#include "inst_f32.inc"
