// FP64 row and column passes for grids with a radix-5, 7 or 11 factor.
#include "kernels_impl.cuh"
HS_INSTANTIATE_EXT(double, 4)
