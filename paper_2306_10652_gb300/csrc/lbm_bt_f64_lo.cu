// Batched-form instantiations: thermodynamics in double, Nc 1..5.
#include "lbm_batch.cuh"
LBM_BT_TU(f64_lo, double, 1, 5)
