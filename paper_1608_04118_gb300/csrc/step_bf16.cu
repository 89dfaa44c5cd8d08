// step_bf16.cu -- step and init kernels with __nv_bfloat16 population storage and float arithmetic.
#include "ltne_step_impl.cuh"
LTNE_DEFINE_LAUNCHERS(bf16, __nv_bfloat16, float)
