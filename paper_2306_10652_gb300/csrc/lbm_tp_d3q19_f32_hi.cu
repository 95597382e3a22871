// Three-pass instantiations: D3Q19, float storage, Nc 9..16.
#include "lbm_threepass.cuh"
LBM_TP_TU(d3q19_f32_hi, 1, float, 9, 16)
