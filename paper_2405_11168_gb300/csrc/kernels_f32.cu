// FP32 instantiations of the solver kernels (column tile: 16 complex = 128 B).
#include "kernels_impl.cuh"
HS_INSTANTIATE(float, false, 16, 256)

