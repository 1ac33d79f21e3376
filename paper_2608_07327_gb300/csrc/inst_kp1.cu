// Row kernels instantiated for padded block width 1.
#define MBPCG_KP 1
#include "inst_kp.inc"
