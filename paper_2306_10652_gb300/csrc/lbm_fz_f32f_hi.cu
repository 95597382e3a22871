// Fused D2Q9 instantiations: storage float, thermodynamics float, Nc 9..16.
#include "lbm_fused2d.cuh"
LBM_FZ_TU(f32f_hi, float, float, 9, 16)
