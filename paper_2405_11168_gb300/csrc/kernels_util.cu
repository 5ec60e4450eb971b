// Small utility kernels: phase-id conversion and validation.
#include "launch.h"

namespace hs {

__global__ void k_ids_u8_to_u16(const uint8_t* in, uint16_t* out, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

__global__ void k_max_id(const uint16_t* ids, size_t n, int* out) {
  int m = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = max(m, (int)ids[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

cudaError_t launch_ids_u8_to_u16(const uint8_t* in, uint16_t* out, size_t n, cudaStream_t s) {
  k_ids_u8_to_u16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

__global__ void k_f32_to_f64(const float* in, double* out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

cudaError_t launch_f32_to_f64(const float* in, double* out, size_t n, cudaStream_t s) {
  k_f32_to_f64<<<1024, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_max_id(const uint16_t* ids, size_t n, int* out, cudaStream_t s) {
  k_max_id<<<1024, 256, 0, s>>>(ids, n, out);
  return cudaGetLastError();
}

}  // namespace hs
