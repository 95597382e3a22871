// Fused D2Q9 instantiations: storage float, thermodynamics double, Nc 9..16.
#include "lbm_fused2d.cuh"
LBM_FZ_TU(f32d_hi, float, double, 9, 16)
