// Row kernels instantiated for padded block width 2.
#define MBPCG_KP 2
#include "inst_kp.inc"
