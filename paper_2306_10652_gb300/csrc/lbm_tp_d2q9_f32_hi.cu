// Three-pass instantiations: D2Q9, float storage, Nc 9..16.
#include "lbm_threepass.cuh"
LBM_TP_TU(d2q9_f32_hi, 0, float, 9, 16)
