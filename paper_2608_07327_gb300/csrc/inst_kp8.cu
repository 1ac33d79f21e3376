// Row kernels instantiated for padded block width 8.
#define MBPCG_KP 8
#include "inst_kp.inc"
