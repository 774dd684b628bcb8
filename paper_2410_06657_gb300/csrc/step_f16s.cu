// Kernels of the f16s storage precision (f in float, h, g, l in __half; arithmetic float; auxiliary fields float).
#include "lbm_launch.cuh"

LBM_DEFINE_LAUNCHERS(f16s, __half, float, float)
LBM_DEFINE_BATCH(f16s, __half, float, float)
