// Three-pass instantiations: D2Q9, double storage, Nc 1..8.
#include "lbm_threepass.cuh"
LBM_TP_TU(d2q9_f64_lo, 0, double, 1, 8)
