// Multi-pass binary32 instantiations: D3Q19, Nc 1..8.
#include "lbm_multipass.cuh"
LBM_MP_TU(d3q19_lo, 1, 1, 8)
