// NTT launchers and kernels for logN = 16 (see ntt_impl.cuh).
#include "ntt_impl.cuh"

FIDES_NTT_DEGREE(16)
