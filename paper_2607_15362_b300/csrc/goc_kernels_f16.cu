// goc_kernels_f16.cu -- the kernels of storage type __half and their launchers.
#include "goc_launch.cuh"

GOC_DEFINE_LAUNCHERS(__half)
