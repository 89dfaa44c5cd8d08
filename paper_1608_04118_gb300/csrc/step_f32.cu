// step_f32.cu -- step and init kernels with float population storage and float arithmetic.
#include "ltne_step_impl.cuh"
LTNE_DEFINE_LAUNCHERS(f32, float, float)
