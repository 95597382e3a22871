// Batched-form instantiations: thermodynamics in double, Nc 6..10.
#include "lbm_batch.cuh"
LBM_BT_TU(f64_hi, double, 6, 10)
