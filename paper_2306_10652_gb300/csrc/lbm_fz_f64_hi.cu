// Fused D2Q9 instantiations: storage double, thermodynamics double, Nc 9..16.
#include "lbm_fused2d.cuh"
LBM_FZ_TU(f64_hi, double, double, 9, 16)
