// Kernels of the f32 storage precision (populations float, arithmetic float, auxiliary fields float).
#include "lbm_launch.cuh"

LBM_DEFINE_LAUNCHERS(f32, float, float, float)
LBM_DEFINE_BATCH(f32, float, float, float)
