// step_f32.cu -- step and init kernels with float population storage and float arithmetic.
#include "ltne_tma.cuh"
LTNE_DEFINE_FLOAT_LAUNCHERS(f32, float)
