// Fused D2Q9 instantiations: storage double, thermodynamics double, Nc 1..8.
#include "lbm_fused2d.cuh"
LBM_FZ_TU(f64_lo, double, double, 1, 8)
