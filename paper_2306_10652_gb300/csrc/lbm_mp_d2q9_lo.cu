// Multi-pass binary32 instantiations: D2Q9, Nc 1..8.
#include "lbm_multipass.cuh"
LBM_MP_TU(d2q9_lo, 0, 1, 8)
