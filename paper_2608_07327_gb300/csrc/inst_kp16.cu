// Row kernels instantiated for padded block width 16.
#define MBPCG_KP 16
#include "inst_kp.inc"
