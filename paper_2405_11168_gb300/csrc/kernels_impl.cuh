// Definitions of the launchers in launch.h; included once per precision.
#pragma once
#include <string.h>

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "launch.h"

namespace hs {

// Raise a kernel's dynamic shared-memory limit when a launch needs more than
// it has been given so far on the current device (the attribute is per device,
// so the record is keyed by device ordinal and kernel).  Launches recorded into
// a graph capture therefore never call the attribute API: the first,
// uncaptured, chunk of a solve has already set it.
inline std::mutex& smem_mu() {
  static std::mutex m;
  return m;
}
inline std::map<std::pair<int, const void*>, size_t>& smem_set() {
  static std::map<std::pair<int, const void*>, size_t> m;
  return m;
}
template <typename K> static cudaError_t set_smem(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const std::pair<int, const void*> key(dev, reinterpret_cast<const void*>(kernel));
  std::lock_guard<std::mutex> lock(smem_mu());
  size_t& have = smem_set()[key];
  if (smem <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) have = smem;
  return e;
}

template <typename T, int TY, class MAT, int MODE, bool REAL, bool BATCH>
static cudaError_t march_launch(const MarchArgs<T>& a, const MAT& m, dim3 g, int nthr, size_t smem,
                                cudaStream_t s) {
  auto k = k_march<T, TY, MAT, MODE, REAL, BATCH>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<g, nthr, smem, s>>>(a, m);
  return cudaGetLastError();
}

// batched launches (zstride != 0) run the real-space force pass only
template <typename T, int TY, class MAT, int MODE, bool REAL>
static cudaError_t march_one(const MarchArgs<T>& a, const MAT& m, dim3 g, int nthr, size_t smem, cudaStream_t s) {
  if constexpr (MODE == MODE_FORCE && REAL) {
    if (a.zstride != 0) return march_launch<T, TY, MAT, MODE, REAL, true>(a, m, g, nthr, smem, s);
  } else {
    if (a.zstride != 0) return cudaErrorInvalidValue;
  }
  return march_launch<T, TY, MAT, MODE, REAL, false>(a, m, g, nthr, smem, s);
}

template <typename T, int TY, bool REAL>
static cudaError_t march_ty(const MarchArgs<T>& a, bool iso, int mode, dim3 g, int nthr, size_t smem,
                            cudaStream_t s) {
  if (mode == MODE_EMIT) {
    if (REAL) return cudaErrorInvalidValue;
    return march_one<T, TY, MatIso<T>, MODE_EMIT, false>(a, MatIso<T>{a.mat}, g, nthr, smem, s);
  }
  if (mode == MODE_FORCE_FIELDS) {  // last FP64 residual sweep of a refined solve
    if constexpr (REAL && sizeof(T) == 8) {
      if (iso) return march_one<T, TY, MatIso<T>, MODE_FORCE_FIELDS, REAL>(a, MatIso<T>{a.mat}, g, nthr, smem, s);
      return march_one<T, TY, MatAniso<T>, MODE_FORCE_FIELDS, REAL>(a, MatAniso<T>{a.mat}, g, nthr, smem, s);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (iso) {
    MatIso<T> m{a.mat};
    if (mode == MODE_FORCE) return march_one<T, TY, MatIso<T>, MODE_FORCE, REAL>(a, m, g, nthr, smem, s);
    return march_one<T, TY, MatIso<T>, MODE_FIELDS, REAL>(a, m, g, nthr, smem, s);
  }
  MatAniso<T> m{a.mat};
  if (mode == MODE_FORCE) return march_one<T, TY, MatAniso<T>, MODE_FORCE, REAL>(a, m, g, nthr, smem, s);
  return march_one<T, TY, MatAniso<T>, MODE_FIELDS, REAL>(a, m, g, nthr, smem, s);
}

// resident blocks per SM of the FP64 real-space force pass (single solves)
template <int TY, class MAT>
static cudaError_t march64_occ_one(int nthr, size_t smem, int* n) {
  auto k = k_march<double, TY, MAT, MODE_FORCE, true, false>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k, nthr, smem);
}
template <int TY>
static cudaError_t march64_occ_ty(bool iso, int nthr, size_t smem, int* n) {
  return iso ? march64_occ_one<TY, MatIso<double>>(nthr, smem, n) : march64_occ_one<TY, MatAniso<double>>(nthr, smem, n);
}

template <typename T, bool REAL>
static cudaError_t march_real(const MarchArgs<T>& a, bool iso, int ty, int mode, dim3 g, int nthr, size_t smem,
                              cudaStream_t s) {
  switch (ty) {
    case 2: return march_ty<T, 2, REAL>(a, iso, mode, g, nthr, smem, s);
    case 4: return march_ty<T, 4, REAL>(a, iso, mode, g, nthr, smem, s);
    case 8: return march_ty<T, 8, REAL>(a, iso, mode, g, nthr, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int TY, class MATP, int MODE, int N1, bool BATCH>
static cudaError_t stencil_launch(const MarchArgs<float>& a, const MATP& m, dim3 g, int nthr, size_t smem,
                                  cudaStream_t s) {
  auto k = k_stencil<TY, MATP, MODE, N1, BATCH>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<g, nthr, smem, s>>>(a, m);
  return cudaGetLastError();
}

// batched launches (zstride != 0) run the force pass only
template <int TY, class MATP, int MODE, int N1 = 0>
static cudaError_t stencil_one(const MarchArgs<float>& a, const MATP& m, dim3 g, int nthr, size_t smem,
                               cudaStream_t s) {
  if constexpr (MODE == MODE_FORCE) {
    if (a.zstride != 0) return stencil_launch<TY, MATP, MODE, N1, true>(a, m, g, nthr, smem, s);
  } else {
    if (a.zstride != 0) return cudaErrorInvalidValue;
  }
  return stencil_launch<TY, MATP, MODE, N1, false>(a, m, g, nthr, smem, s);
}

template <int TY>
static cudaError_t stencil_ty(const MarchArgs<float>& a, bool iso, int mode, dim3 g, int nthr, size_t smem,
                              cudaStream_t s) {
  if (iso) {
    MatIsoP m{a.mat};
    if constexpr (TY == 4) {
      if (mode == MODE_FORCE && a.n1 == 256 && nthr == 256)
        return stencil_one<TY, MatIsoP, MODE_FORCE, 256>(a, m, g, nthr, smem, s);
    }
    if (mode == MODE_FORCE) return stencil_one<TY, MatIsoP, MODE_FORCE>(a, m, g, nthr, smem, s);
    return stencil_one<TY, MatIsoP, MODE_FIELDS>(a, m, g, nthr, smem, s);
  }
  MatAnisoP m{a.mat};
  if constexpr (TY == 4) {
    if (mode == MODE_FORCE && a.n1 == 256 && nthr == 256)
      return stencil_one<TY, MatAnisoP, MODE_FORCE, 256>(a, m, g, nthr, smem, s);
  }
  if (mode == MODE_FORCE) return stencil_one<TY, MatAnisoP, MODE_FORCE>(a, m, g, nthr, smem, s);
  return stencil_one<TY, MatAnisoP, MODE_FIELDS>(a, m, g, nthr, smem, s);
}

// FP32 real-space pass (FORCE / FIELDS on a real displacement field); a
// template so that only the unit that launches it instantiates its kernels
template <int UNUSED = 0>
static cudaError_t stencil_f32(const MarchArgs<float>& a, bool iso, int ty, int mode, dim3 g, int nthr,
                               size_t smem, cudaStream_t s) {
  if (mode != MODE_FORCE && mode != MODE_FIELDS) return cudaErrorInvalidValue;
  switch (ty) {
    case 2: return stencil_ty<2>(a, iso, mode, g, nthr, smem, s);
    case 4: return stencil_ty<4>(a, iso, mode, g, nthr, smem, s);
    case 8: return stencil_ty<8>(a, iso, mode, g, nthr, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int CT, int MODE, int LF = 0, int NT = 0>
static cudaError_t col_one(const ColArgs<T>& a, dim3 g, int nthr, size_t smem, cudaStream_t s) {
  auto k = k_col<T, CT, MODE, LF, NT>;
  if constexpr (MODE == COL_Z_GREEN && LF > 0) {
    if (a.tma && !a.state_smem) k = k_col<T, CT, MODE, LF, NT, true>;
  }
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<g, nthr, smem, s>>>(a);
  return cudaGetLastError();
}

// real-displacement passes: the packed FP32 kernel, or k_march for FP64
template <typename T>
static cudaError_t march_real_dispatch(const MarchArgs<T>& a, bool iso, int ty, int mode, dim3 g, int nthr,
                                      size_t smem, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) return stencil_f32<>(a, iso, ty, mode, g, nthr, smem, s);
  else return march_real<double, true>(a, iso, ty, mode, g, nthr, smem, s);
}

template <typename T, int CT, int LF = 0, int NT = 0>
static cudaError_t col_ct(const ColArgs<T>& a, int mode, dim3 g, int nthr, size_t smem, cudaStream_t s) {
  switch (mode) {
    case COL_Y_FWD: return col_one<T, CT, COL_Y_FWD, LF, NT>(a, g, nthr, smem, s);
    case COL_Y_INV: return col_one<T, CT, COL_Y_INV, LF, NT>(a, g, nthr, smem, s);
    case COL_Z_GREEN: return col_one<T, CT, COL_Z_GREEN, LF, NT>(a, g, nthr, smem, s);
    case COL_Z_INV_STATE: return col_one<T, CT, COL_Z_INV_STATE, LF, NT>(a, g, nthr, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

// transformed length of a column pass
template <typename T> static int col_length(const ColArgs<T>& a, int mode) {
  return (mode == COL_Y_FWD || mode == COL_Y_INV) ? a.n2 : a.n3;
}

// compile-time variants for the default tile and block size at the hot lengths
template <typename T, int CT, int NT>
static cudaError_t col_dispatch(const ColArgs<T>& a, int mode, dim3 g, int nthr, size_t smem, cudaStream_t s) {
  const int L = col_length(a, mode);
  if (nthr == NT) {
    if (L == 256) return col_ct<T, CT, 256, NT>(a, mode, g, nthr, smem, s);
    if (L == 512) return col_ct<T, CT, 512, NT>(a, mode, g, nthr, smem, s);
    if (L == 128) return col_ct<T, CT, 128, NT>(a, mode, g, nthr, smem, s);
    if (L == 64) return col_ct<T, CT, 64, NT>(a, mode, g, nthr, smem, s);
  }
  return col_ct<T, CT>(a, mode, g, nthr, smem, s);
}

template <typename T, int CT, int MODE, int LF, int NT>
static cudaError_t colp_one(const ColArgs<T>& a, dim3 g, size_t smem, cudaStream_t s, int* occ) {
  auto k = k_colp<T, CT, MODE, LF, NT>;
  if (a.tma) k = k_colp<T, CT, MODE, LF, NT, true>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  if (occ != nullptr) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, NT, smem);
  k<<<g, NT, smem, s>>>(a);
  return cudaGetLastError();
}

// the persistent column pass at a fixed length: launch it, or (occ) its blocks per SM
template <typename T, int CT, int NT, int LF>
static cudaError_t colp_mode(const ColArgs<T>& a, int mode, dim3 g, size_t smem, cudaStream_t s, int* occ) {
  switch (mode) {
    case COL_Y_FWD: return colp_one<T, CT, COL_Y_FWD, LF, NT>(a, g, smem, s, occ);
    case COL_Y_INV: return colp_one<T, CT, COL_Y_INV, LF, NT>(a, g, smem, s, occ);
    case COL_Z_GREEN: return colp_one<T, CT, COL_Z_GREEN, LF, NT>(a, g, smem, s, occ);
    default: return cudaErrorNotSupported;
  }
}

template <typename T, int CT, int NT>
static cudaError_t colp_dispatch(const ColArgs<T>& a, int mode, int L, dim3 g, int nthr, size_t smem,
                                 cudaStream_t s, int* occ) {
  if (nthr != NT) return cudaErrorNotSupported;
  switch (L) {
    case 64: return colp_mode<T, CT, NT, 64>(a, mode, g, smem, s, occ);
    case 128: return colp_mode<T, CT, NT, 128>(a, mode, g, smem, s, occ);
    case 256: return colp_mode<T, CT, NT, 256>(a, mode, g, smem, s, occ);
    case 512: return colp_mode<T, CT, NT, 512>(a, mode, g, smem, s, occ);
    default: return cudaErrorNotSupported;
  }
}

template <typename T, int MODE, int LF, bool BATCH>
static cudaError_t row_launch(const RowArgs<T>& a, dim3 nb, int nthr, size_t smem, cudaStream_t s) {
  auto k = k_row<T, MODE, LF, BATCH>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<nb, nthr, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int MODE, int LF = 0>
static cudaError_t row_one(const RowArgs<T>& a, dim3 nb, int nthr, size_t smem, cudaStream_t s) {
  if (a.zstride != 0) return row_launch<T, MODE, LF, true>(a, nb, nthr, smem, s);
  return row_launch<T, MODE, LF, false>(a, nb, nthr, smem, s);
}

template <typename T, int MODE, int LF = 0>
static cudaError_t row_occ_one(int nthr, size_t smem, int* n) {
  auto k = k_row<T, MODE, LF>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k, nthr, smem);
}

template <typename T, int MODE>
static cudaError_t row_occ(int n1, int nthr, size_t smem, int* n) {
  if (nthr == 256) {
    if (n1 == 256) return row_occ_one<T, MODE, 256>(nthr, smem, n);
    if (n1 == 512) return row_occ_one<T, MODE, 512>(nthr, smem, n);
    if (n1 == 128) return row_occ_one<T, MODE, 128>(nthr, smem, n);
    if (n1 == 64) return row_occ_one<T, MODE, 64>(nthr, smem, n);
  }
  return row_occ_one<T, MODE>(nthr, smem, n);
}

// compile-time variants for 256-thread blocks at the hot lengths
template <typename T, int MODE>
static cudaError_t row_dispatch(const RowArgs<T>& a, dim3 nb, int nthr, size_t smem, cudaStream_t s) {
  if (nthr == 256) {
    if (a.n1 == 256) return row_one<T, MODE, 256>(a, nb, nthr, smem, s);
    if (a.n1 == 512) return row_one<T, MODE, 512>(a, nb, nthr, smem, s);
    if (a.n1 == 128) return row_one<T, MODE, 128>(a, nb, nthr, smem, s);
    if (a.n1 == 64) return row_one<T, MODE, 64>(a, nb, nthr, smem, s);
  }
  return row_one<T, MODE>(a, nb, nthr, smem, s);
}

template <typename T>
__global__ void k_state_export(const typename cplx_t<T>::type* S, double2* out, size_t nrows, int nh, int P) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows * nh) return;
  size_t r = i / nh, k = i - r * nh;
  auto v = S[r * P + k];
  out[i] = make_double2((double)v.x, (double)v.y);
}

template <typename T>
__global__ void k_state_import(const double2* in, typename cplx_t<T>::type* S, size_t nrows, int nh, int P) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows * P) return;
  size_t r = i / P, k = i - r * P;
  typename cplx_t<T>::type v;
  if ((int)k < nh) {
    double2 d = in[r * nh + k];
    v.x = (T)d.x;
    v.y = (T)d.y;
  } else {
    v.x = 0;
    v.y = 0;
  }
  S[i] = v;
}

}  // namespace hs

// CT: the wider column tile (CT / 2 is the default); NT: the default
// column-pass block size, which gets compile-time variants at hot lengths.
#define HS_INSTANTIATE(T, REALOK, CT, NT)                                                                 \
  namespace hs {                                                                                         \
  template <>                                                                                            \
  cudaError_t launch_march<T>(const MarchArgs<T>& a, bool iso, int ty, int mode, bool real, dim3 grid,  \
                              int nthr, size_t smem, cudaStream_t s) {                                   \
    if (a.ids == nullptr || a.mat == nullptr || a.st == nullptr || a.partials == nullptr)                \
      return cudaErrorInvalidValue;                                                                      \
    if (real && a.ureal == nullptr) return cudaErrorInvalidValue;                                        \
    if (!real && a.in == nullptr) return cudaErrorInvalidValue;                                          \
    if (mode == MODE_EMIT && a.u64 == nullptr) return cudaErrorInvalidValue;                             \
    if (mode == MODE_FORCE && !real && a.out == nullptr) return cudaErrorInvalidValue;                   \
    if ((mode == MODE_FIELDS || mode == MODE_FORCE_FIELDS) && (a.eps_out == nullptr || a.sig_out == nullptr)) \
      return cudaErrorInvalidValue;                                                                      \
    if (real) return march_real_dispatch(a, iso, ty, mode, grid, nthr, smem, s);                         \
    return march_real<T, false>(a, iso, ty, mode, grid, nthr, smem, s);                                  \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t launch_col<T>(const ColArgs<T>& a, int mode, int ct, dim3 grid, int nthr, size_t smem,      \
                            cudaStream_t s) {                                                            \
    if (a.buf == nullptr || a.tw == nullptr || ((mode == COL_Z_GREEN || mode == COL_Z_INV_STATE) && a.S == nullptr)) \
      return cudaErrorInvalidValue;                                                                      \
    if (plan_ext(a.plan)) return launch_col_ext<T>(a, mode, ct, grid, nthr, smem, s);                  \
    if (ct == (CT)) return col_ct<T, CT>(a, mode, grid, nthr, smem, s);                                  \
    if (ct == (CT) / 2) return col_dispatch<T, (CT) / 2, NT>(a, mode, grid, nthr, smem, s);              \
    return cudaErrorInvalidValue;                                                                        \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t launch_colp<T>(const ColArgs<T>& a, int mode, int ct, dim3 grid, int nthr, size_t smem,     \
                             cudaStream_t s) {                                                           \
    if (a.buf == nullptr || a.tw == nullptr || (mode == COL_Z_GREEN && a.S == nullptr))                  \
      return cudaErrorInvalidValue;                                                                      \
    if (ct != (CT) / 2 || plan_ext(a.plan) || a.state_smem) return cudaErrorNotSupported;               \
    return colp_dispatch<T, (CT) / 2, NT>(a, mode, col_length(a, mode), grid, nthr, smem, s, nullptr);   \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t march_blocks_per_sm<T>(bool iso, int ty, int nthr, size_t smem, int* n) {                 \
    if (sizeof(T) != 8) return cudaErrorNotSupported;                                                    \
    switch (ty) {                                                                                        \
      case 2: return march64_occ_ty<2>(iso, nthr, smem, n);                                              \
      case 4: return march64_occ_ty<4>(iso, nthr, smem, n);                                              \
      case 8: return march64_occ_ty<8>(iso, nthr, smem, n);                                              \
      default: return cudaErrorInvalidValue;                                                             \
    }                                                                                                    \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t colp_blocks_per_sm<T>(int mode, int L, int ct, int nthr, size_t smem, int* n) {            \
    if (ct != (CT) / 2) return cudaErrorNotSupported;                                                    \
    ColArgs<T> a;                                                                                        \
    memset(&a, 0, sizeof(a));                                                                            \
    return colp_dispatch<T, (CT) / 2, NT>(a, mode, L, dim3(1), nthr, smem, nullptr, n);                  \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t launch_row<T>(const RowArgs<T>& a, int mode, dim3 nb, int nthr, size_t smem, cudaStream_t s) { \
    if (a.tw == nullptr || (mode == ROW_C2R ? (a.spec_in == nullptr || (a.real_out == nullptr && a.acc64 == nullptr)) \
                                            : (a.real_in == nullptr || a.spec_out == nullptr)))         \
      return cudaErrorInvalidValue;                                                                      \
    if (plan_ext(a.plan)) return launch_row_ext<T>(a, mode, nb, nthr, smem, s);                        \
    return mode == ROW_C2R ? row_dispatch<T, ROW_C2R>(a, nb, nthr, smem, s)                             \
                           : row_dispatch<T, ROW_R2C>(a, nb, nthr, smem, s);                            \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t row_blocks_per_sm<T>(int mode, int n1, int nthr, size_t smem, int* n) {                     \
    if (n1 % 5 == 0 || n1 % 7 == 0 || n1 % 11 == 0) return row_blocks_per_sm_ext<T>(mode, nthr, smem, n);  \
    return mode == ROW_C2R ? row_occ<T, ROW_C2R>(n1, nthr, smem, n) : row_occ<T, ROW_R2C>(n1, nthr, smem, n); \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t launch_state_export<T>(const typename cplx_t<T>::type* S, double2* out, int n2, int n3,     \
                                     int nh, int P, cudaStream_t s) {                                    \
    size_t nrows = (size_t)3 * n3 * n2, n = nrows * nh;                                                  \
    k_state_export<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S, out, nrows, nh, P);                 \
    return cudaGetLastError();                                                                           \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t launch_state_import<T>(const double2* in, typename cplx_t<T>::type* S, int n2, int n3,      \
                                     int nh, int P, cudaStream_t s) {                                    \
    size_t nrows = (size_t)3 * n3 * n2, n = nrows * P;                                                   \
    k_state_import<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, S, nrows, nh, P);                  \
    return cudaGetLastError();                                                                           \
  }                                                                                                      \
  }

// Kernels for plans with a radix-5, 7 or 11 stage, in their own translation unit.
#define HS_INSTANTIATE_EXT(T, CT)                                                                         \
  namespace hs {                                                                                         \
  template <>                                                                                            \
  cudaError_t launch_col_ext<T>(const ColArgs<T>& a, int mode, int ct, dim3 grid, int nthr, size_t smem, \
                                cudaStream_t s) {                                                        \
    if (ct != (CT)) return cudaErrorInvalidValue;                                                        \
    return col_ct<T, CT, -1>(a, mode, grid, nthr, smem, s);                                              \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t launch_row_ext<T>(const RowArgs<T>& a, int mode, dim3 nb, int nthr, size_t smem, cudaStream_t s) { \
    return mode == ROW_C2R ? row_one<T, ROW_C2R, -1>(a, nb, nthr, smem, s)                               \
                           : row_one<T, ROW_R2C, -1>(a, nb, nthr, smem, s);                              \
  }                                                                                                      \
  template <>                                                                                            \
  cudaError_t row_blocks_per_sm_ext<T>(int mode, int nthr, size_t smem, int* n) {                        \
    return mode == ROW_C2R ? row_occ_one<T, ROW_C2R, -1>(nthr, smem, n)                                  \
                           : row_occ_one<T, ROW_R2C, -1>(nthr, smem, n);                                 \
  }                                                                                                      \
  }
