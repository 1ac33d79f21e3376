// Row kernels instantiated for padded block width 4.
#define MBPCG_KP 4
#include "inst_kp.inc"
