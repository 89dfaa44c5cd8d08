// step_f16.cu -- step and init kernels with __half population storage and float arithmetic.
#include "ltne_step_impl.cuh"
LTNE_DEFINE_LAUNCHERS(f16, __half, float)
