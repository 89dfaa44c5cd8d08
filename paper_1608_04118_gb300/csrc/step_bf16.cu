// step_bf16.cu -- step and init kernels with __nv_bfloat16 population storage and float arithmetic.
#include "ltne_tma.cuh"
LTNE_DEFINE_FLOAT_LAUNCHERS(bf16, __nv_bfloat16)
