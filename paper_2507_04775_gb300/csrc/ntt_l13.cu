// NTT launchers and kernels for logN = 13 (see ntt_impl.cuh).
#include "ntt_impl.cuh"

FIDES_NTT_DEGREE(13)
