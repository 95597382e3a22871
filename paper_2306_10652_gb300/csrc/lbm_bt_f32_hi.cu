// Batched-form instantiations: thermodynamics in float, Nc 6..10.
#include "lbm_batch.cuh"
LBM_BT_TU(f32_hi, float, 6, 10)
