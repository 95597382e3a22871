// Fused D2Q9 instantiations: storage float, thermodynamics double-binary32, Nc 9..16.
#include "lbm_fused2d.cuh"
LBM_FZ_TU(f32d_hi, float, DF64, 9, 16)
