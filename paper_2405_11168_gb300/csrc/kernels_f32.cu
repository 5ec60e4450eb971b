// FP32 instantiations of the solver kernels (column tile: 16 complex = 128 B), and the
// column-pair real-space pass of the FP32 iterations.
#include "kernels_impl.cuh"
HS_INSTANTIATE(float, false, 16, 256)

namespace hs {

template <int TY, class MAT>
static cudaError_t xpair_one(const XpArgs& a, const MAT& m, dim3 g, int nthr, size_t smem, cudaStream_t s) {
  auto k = k_xpair<TY, MAT>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<g, nthr, smem, s>>>(a, m);
  return cudaGetLastError();
}

cudaError_t launch_xpair(const XpArgs& a, bool iso, int ty, dim3 grid, int nthr, size_t smem, cudaStream_t s) {
  if (a.ureal == nullptr || a.ids == nullptr || a.mat == nullptr || a.fout == nullptr || a.side == nullptr ||
      a.partials == nullptr || a.st == nullptr || ty != 1 || (a.n1 & 1) != 0)
    return cudaErrorInvalidValue;
  if (iso) return xpair_one<1>(a, XpIso{a.mat}, grid, nthr, smem, s);
  return xpair_one<1>(a, XpAniso{a.mat}, grid, nthr, smem, s);
}

cudaError_t xpair_blocks_per_sm(bool iso, int ty, int nthr, size_t smem, int* n) {
  if (ty != 1) return cudaErrorInvalidValue;
  cudaError_t e;
  if (iso) {
    e = set_smem(k_xpair<1, XpIso>, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_xpair<1, XpIso>, nthr, smem);
  } else {
    e = set_smem(k_xpair<1, XpAniso>, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_xpair<1, XpAniso>, nthr, smem);
  }
  return e;
}

}  // namespace hs
