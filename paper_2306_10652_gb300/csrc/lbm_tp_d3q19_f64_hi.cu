// Three-pass instantiations: D3Q19, double storage, Nc 9..16.
#include "lbm_threepass.cuh"
LBM_TP_TU(d3q19_f64_hi, 1, double, 9, 16)
