// Three-pass instantiations: D3Q19, double storage, Nc 1..8.
#include "lbm_threepass.cuh"
LBM_TP_TU(d3q19_f64_lo, 1, double, 1, 8)
