// Instantiations of the mu / force evaluation (lbm_forces), Nc 9..16.
#include "lbm_fields.cuh"
LBM_FIELDS_TU(launch_forces_hi, 9, 16)
