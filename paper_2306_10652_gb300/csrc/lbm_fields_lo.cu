// Instantiations of the mu / force evaluation (lbm_forces), Nc 1..8.
#include "lbm_fields.cuh"
LBM_FIELDS_TU(launch_forces_lo, 1, 8)
