// Three-pass instantiations: D3Q19, float storage, Nc 1..8.
#include "lbm_threepass.cuh"
LBM_TP_TU(d3q19_f32_lo, 1, float, 1, 8)
