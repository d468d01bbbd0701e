// goc_kernels_f32.cu -- the kernels of storage type float and their launchers.
#include "goc_launch.cuh"

GOC_DEFINE_LAUNCHERS(float)
