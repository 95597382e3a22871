// Fused D2Q9 instantiations: storage float, thermodynamics double, Nc 1..8.
#include "lbm_fused2d.cuh"
LBM_FZ_TU(f32d_lo, float, double, 1, 8)
