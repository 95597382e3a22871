// Batched-form instantiations: thermodynamics in float, Nc 1..5.
#include "lbm_batch.cuh"
LBM_BT_TU(f32_lo, float, 1, 5)
