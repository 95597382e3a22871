// Fused D2Q9 instantiations: storage float, thermodynamics double-binary32, Nc 1..8.
#include "lbm_fused2d.cuh"
LBM_FZ_TU(f32d_lo, float, DF64, 1, 8)
