// Fused D2Q9 instantiations: storage float, thermodynamics float, Nc 1..8.
#include "lbm_fused2d.cuh"
LBM_FZ_TU(f32f_lo, float, float, 1, 8)
