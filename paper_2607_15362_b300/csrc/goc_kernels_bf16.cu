// goc_kernels_bf16.cu -- the kernels of storage type __nv_bfloat16 and their launchers.
#include "goc_launch.cuh"

GOC_DEFINE_LAUNCHERS(__nv_bfloat16)
