// Multi-pass binary32 instantiations: D2Q9, Nc 9..16.
#include "lbm_multipass.cuh"
LBM_MP_TU(d2q9_hi, 0, 9, 16)
