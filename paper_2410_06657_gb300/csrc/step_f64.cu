// Kernels of the f64 storage precision (populations double, arithmetic double, auxiliary fields double).
#include "lbm_launch.cuh"

LBM_DEFINE_LAUNCHERS(f64, double, double, double)
LBM_DEFINE_BATCH(f64, double, double, double)
