// step_f16.cu -- step and init kernels with __half population storage and float arithmetic.
#include "ltne_tma.cuh"
LTNE_DEFINE_FLOAT_LAUNCHERS(f16, __half)
