// Three-pass instantiations: D2Q9, float storage, Nc 1..8.
#include "lbm_threepass.cuh"
LBM_TP_TU(d2q9_f32_lo, 0, float, 1, 8)
