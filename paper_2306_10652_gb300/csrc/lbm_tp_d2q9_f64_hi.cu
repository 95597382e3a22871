// Three-pass instantiations: D2Q9, double storage, Nc 9..16.
#include "lbm_threepass.cuh"
LBM_TP_TU(d2q9_f64_hi, 0, double, 9, 16)
