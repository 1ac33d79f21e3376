// Row kernels instantiated for padded block width 32.
#define MBPCG_KP 32
#include "inst_kp.inc"
