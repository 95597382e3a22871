// Multi-pass binary32 instantiations: D3Q19, Nc 9..16.
#include "lbm_multipass.cuh"
LBM_MP_TU(d3q19_hi, 1, 9, 16)
