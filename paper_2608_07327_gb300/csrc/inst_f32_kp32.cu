// FP32 row kernels of the mixed-precision inner solve, padded block width 32.
#define MBPCG_KP 32
#include "inst_f32.inc"
