// Internal launch interface between the C-ABI host code and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "colpass.cuh"
#include "march.cuh"
#include "rowpass.cuh"
#include "stencil.cuh"

namespace hs {

// mode: MODE_FORCE / MODE_FIELDS / MODE_EMIT; real: input is the FP64 real
// displacement field (only for T = double).
template <typename T>
cudaError_t launch_march(const MarchArgs<T>& a, bool iso, int ty, int mode, bool real, dim3 grid, int nthr,
                         size_t smem, cudaStream_t s);

template <typename T>
cudaError_t launch_col(const ColArgs<T>& a, int mode, int ct, dim3 grid, int nthr, size_t smem, cudaStream_t s);

// persistent double-buffered column pass (COL_Y_FWD, COL_Y_INV, COL_Z_GREEN) for the compile-time
// lengths 64, 128, 256, 512 with the default tile and block size: grid.x persistent blocks,
// grid.z items; cudaErrorNotSupported when no such variant exists
template <typename T>
cudaError_t launch_colp(const ColArgs<T>& a, int mode, int ct, dim3 grid, int nthr, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t colp_blocks_per_sm(int mode, int L, int ct, int nthr, size_t smem, int* n);

// resident blocks per SM of the FP64 real-space force pass of a single solve (T = double only)
template <typename T>
cudaError_t march_blocks_per_sm(bool iso, int ty, int nthr, size_t smem, int* n);

// mode: ROW_C2R / ROW_R2C; grid.x persistent blocks per item, grid.z items (batched launches)
template <typename T>
cudaError_t launch_row(const RowArgs<T>& a, int mode, dim3 grid, int nthr, size_t smem, cudaStream_t s);

// the same passes for plans with a radix-5, 7 or 11 stage (default column tile only)
template <typename T>
cudaError_t launch_col_ext(const ColArgs<T>& a, int mode, int ct, dim3 grid, int nthr, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_row_ext(const RowArgs<T>& a, int mode, dim3 grid, int nthr, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t row_blocks_per_sm_ext(int mode, int nthr, size_t smem, int* n);

// resident blocks per SM of the row pass (persistent grid sizing)
template <typename T>
cudaError_t row_blocks_per_sm(int mode, int n1, int nthr, size_t smem, int* n);

// u8 phase ids -> u16
cudaError_t launch_ids_u8_to_u16(const uint8_t* in, uint16_t* out, size_t n, cudaStream_t s);
// widen a float array to double
cudaError_t launch_f32_to_f64(const float* in, double* out, size_t n, cudaStream_t s);
// largest id into *out (int, must start at 0)
cudaError_t launch_max_id(const uint16_t* ids, size_t n, int* out, cudaStream_t s);
// padded T-complex state <-> packed complex128 [3][n3][n2][nh]
template <typename T>
cudaError_t launch_state_export(const typename cplx_t<T>::type* S, double2* out, int n2, int n3, int nh, int P,
                                cudaStream_t s);
template <typename T>
cudaError_t launch_state_import(const double2* in, typename cplx_t<T>::type* S, int n2, int n3, int nh, int P,
                                cudaStream_t s);

}  // namespace hs
