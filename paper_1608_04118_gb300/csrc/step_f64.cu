// step_f64.cu -- step and init kernels with double population storage and double arithmetic.
#include "ltne_step_impl.cuh"
LTNE_DEFINE_LAUNCHERS(f64, double, double)
