// FP64 instantiations of the solver kernels (column tile: 8 complex = 128 B),
// including the real-space FP64 residual sweep used by the refined mode.
#include "kernels_impl.cuh"
HS_INSTANTIATE(double, true, 8, 128)
