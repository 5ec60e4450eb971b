// Column passes: FFTs along y or z of the half-spectrum fields, and the Green
// update fused between the forward and inverse z transforms.
//
// A block owns CT consecutive x-frequency columns (one 128-byte row segment
// per component) of one z (y-pass) or one y (z-pass) and all three
// displacement/force components.  Shared-memory layout [e][comp][col], so
// every row of the tile is contiguous and each FFT sequence is a column.
//
// Green update (Algorithm 1 step 5, with Eq. Green_tensor): at every q,
//   Dt_i(q) = D_i(q) exp(-i q.(1/2,1/2,1/2)) from the per-axis tables
//            exp(-i q_x), exp(-i q_y), exp(-i q_z) (corner-indexed state),
//   M_ik = 2 Re(Dt_i conj(Dt_k)),  Omega^-1_jl = sum_ik lambda0_jikl M_ik,
//   u(q) <- u(q) - (2/N) Omega(q) F_unnormalised(q),
// with Omega = 0 and u = 0 at q = 0 and q = (pi,pi,pi) (Section 2.3).
// The factor 2 is f = 2 F_hat (the force transform equals half the
// equilibrium residual f of Eq. basic_scheme_dep_2); 1/N is the forward
// normalisation of Eq. FT, applied here once.
#pragma once
#include <cuda.h>  // CUtensorMap (the descriptor type only; no driver call from device code)

#include "common.cuh"

namespace hs {

enum { COL_Y_FWD = 0, COL_Y_INV = 1, COL_Z_GREEN = 2, COL_Z_INV_STATE = 3 };
// dynamic shared memory a TMA-fed persistent column pass needs beyond its two tiles (alignment
// of the tiles to 128 bytes, two mbarriers)
constexpr size_t kColpTmaSlack = 256;

template <typename T> struct ColArgs {
  using C = typename cplx_t<T>::type;
  C* buf;            // [3][n3][n2][P]
  C* S;              // state u_hat, same layout
  const C* tw;       // w_L^j of the transformed axis
  const C* tw1;      // exp(-i q_x) table (= w_N1^h)
  const C* tw2;
  const C* tw3;
  FftPlan plan;
  int n1, n2, n3, P, nh;
  T scale;           // 2/N
  T G6[36];          // Omega^-1 (Voigt pairs) = G6 . M (Voigt pairs)
  // isotropic reference medium: Omega^-1 = c0a M + c0b tr(M) I with c0a = lambda0 + mu0,
  // c0b = mu0 (used when c0iso != 0, or always when c0dev is given)
  int c0iso;
  T c0a, c0b;
  const T* c0dev;    // not null: (c0a, c0b) read here (per item in batched launches)
  DevStatus* st;
  int skip_if_done;
  size_t zstride;    // batched launches: bytes between the workspaces of consecutive items
  int state_smem;    // COL_Z_GREEN: 1 = the state tile is copied to shared memory beside the force
                     // tile (its copy overlaps the forward transform); 0 = read point by point
  int tma;           // persistent y passes and the fixed-length z pass: tiles loaded by tensor
                     // copies described by tmap
  // rank-5 tiled map of buf as T elements: (2P x-values, 3 components, n2, n3, items), box
  // (2 CT, 3, min(n2, 256), 1, 1) for the y passes or (2 CT, 3, 1, min(n3, 256), 1) for the z
  // pass; the component dimension sits inside y so that a box lands as the [e][comp][col] tile
  CUtensorMap tmap;
};

template <typename T> __device__ __forceinline__ ColArgs<T> col_item_args(const ColArgs<T>& a) {
  if (a.zstride == 0) return a;
  ColArgs<T> b = a;
  const size_t o = (size_t)blockIdx.z * a.zstride;
  b.buf = zshift(a.buf, o);
  b.S = zshift(a.S, o);
  b.tw = zshift(a.tw, o);
  b.tw1 = zshift(a.tw1, o);
  b.tw2 = zshift(a.tw2, o);
  b.tw3 = zshift(a.tw3, o);
  b.c0dev = zshift(a.c0dev, o);
  b.st = zshift(a.st, o);
  return b;
}

template <typename T>
__device__ __forceinline__ void green_core(const ColArgs<T>& a, T c0a, T c0b, bool c0iso,
                                           typename cplx_t<T>::type yz, typename cplx_t<T>::type xy,
                                           typename cplx_t<T>::type xz, typename cplx_t<T>::type (&F)[3],
                                           typename cplx_t<T>::type (&U)[3]);

// The Green update's arithmetic with every rounding spelled out (a product rounded on its own,
// or fused into one FMA), so that its results do not depend on how the compiler contracts the
// expressions in the kernel it is inlined into: every column-pass variant gives the same bits.
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }
__device__ __forceinline__ float fma_rn(float x, float y, float z) { return __fmaf_rn(x, y, z); }
__device__ __forceinline__ double fma_rn(double x, double y, double z) { return __fma_rn(x, y, z); }
template <typename C> __device__ __forceinline__ C cmul_rn(C p, C q) {
  return cmk<C>(fma_rn(p.x, q.x, -mul_rn(p.y, q.y)), fma_rn(p.x, q.y, mul_rn(p.y, q.x)));
}

template <typename T>
__device__ __forceinline__ void green_apply(const ColArgs<T>& a, T c0a, T c0b, bool c0iso, int h1, int h2, int h3,
                                            typename cplx_t<T>::type (&F)[3],
                                            typename cplx_t<T>::type (&U)[3]) {
  using C = typename cplx_t<T>::type;
  const bool trans = (h1 == 0 && h2 == 0 && h3 == 0) ||
                     (2 * h1 == a.n1 && 2 * h2 == a.n2 && 2 * h3 == a.n3);
  if (trans) {
#pragma unroll
    for (int j = 0; j < 3; ++j) U[j] = cmk<C>(0, 0);
    return;
  }
  const C ex = __ldg(a.tw1 + h1), ey = __ldg(a.tw2 + h2), ez = __ldg(a.tw3 + h3);
  green_core<T>(a, c0a, c0b, c0iso, cmul_rn(ey, ez), cmul_rn(ex, ey), cmul_rn(ex, ez), F, U);
}

// The update at one q from the products of the per-axis phase factors exp(-i q_y) exp(-i q_z)
// (yz), exp(-i q_x) exp(-i q_y) (xy) and exp(-i q_x) exp(-i q_z) (xz); q not a translation mode.
template <typename T>
__device__ __forceinline__ void green_core(const ColArgs<T>& a, T c0a, T c0b, bool c0iso,
                                           typename cplx_t<T>::type yz, typename cplx_t<T>::type xy,
                                           typename cplx_t<T>::type xz, typename cplx_t<T>::type (&F)[3],
                                           typename cplx_t<T>::type (&U)[3]) {
  using C = typename cplx_t<T>::type;
  // corner-convention symbols (Eq. Dq times exp(-i q.(1/2,1/2,1/2))), here 2 D
  C D[3];
  D[0] = cmk<C>(T(1) + yz.x - xy.x - xz.x, yz.y - xy.y - xz.y);
  D[1] = cmk<C>(T(1) - yz.x - xy.x + xz.x, -yz.y - xy.y + xz.y);
  D[2] = cmk<C>(T(1) - yz.x + xy.x - xz.x, -yz.y + xy.y - xz.y);
  // 2 M in Voigt pair order (11,22,33,23,13,12), M_ik = 2 Re(D_i conj D_k); the factors of two
  // are powers of two, so folding them into the constants below changes no rounding
  T M[6];
  M[0] = fma_rn(D[0].x, D[0].x, mul_rn(D[0].y, D[0].y));
  M[1] = fma_rn(D[1].x, D[1].x, mul_rn(D[1].y, D[1].y));
  M[2] = fma_rn(D[2].x, D[2].x, mul_rn(D[2].y, D[2].y));
  M[3] = fma_rn(D[1].x, D[2].x, mul_rn(D[1].y, D[2].y));
  M[4] = fma_rn(D[0].x, D[2].x, mul_rn(D[0].y, D[2].y));
  M[5] = fma_rn(D[0].x, D[1].x, mul_rn(D[0].y, D[1].y));
  T A[6];
  if (c0iso) {
    // Omega^-1_jl = sum_ik lambda0_jikl M_ik = (lambda0 + mu0) M_jl + mu0 tr(M) delta_jl
    const T tr = mul_rn(T(0.5) * c0b, (M[0] + M[1] + M[2]));
    const T ca = T(0.5) * c0a;
#pragma unroll
    for (int i = 0; i < 6; ++i) A[i] = i < 3 ? fma_rn(ca, M[i], tr) : mul_rn(ca, M[i]);
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      T s = mul_rn(a.G6[i * 6], M[0]);
#pragma unroll
      for (int j = 1; j < 6; ++j) s = fma_rn(a.G6[i * 6 + j], M[j], s);
      A[i] = T(0.5) * s;
    }
  }
  // inverse of the symmetric 3x3 [[A0,A5,A4],[A5,A1,A3],[A4,A3,A2]]
  const T c11 = fma_rn(A[1], A[2], -mul_rn(A[3], A[3]));
  const T c22 = fma_rn(A[0], A[2], -mul_rn(A[4], A[4]));
  const T c33 = fma_rn(A[0], A[1], -mul_rn(A[5], A[5]));
  const T c23 = fma_rn(A[4], A[5], -mul_rn(A[0], A[3]));
  const T c13 = fma_rn(A[5], A[3], -mul_rn(A[1], A[4]));
  const T c12 = fma_rn(A[4], A[3], -mul_rn(A[2], A[5]));
  const T det = fma_rn(A[4], c13, fma_rn(A[5], c12, mul_rn(A[0], c11)));
  const T s = a.scale / det;
  const T O[3][3] = {{mul_rn(c11, s), mul_rn(c12, s), mul_rn(c13, s)},
                     {mul_rn(c12, s), mul_rn(c22, s), mul_rn(c23, s)},
                     {mul_rn(c13, s), mul_rn(c23, s), mul_rn(c33, s)}};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    C acc = U[j];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc.x = fma_rn(-O[j][k], F[k].x, acc.x);
      acc.y = fma_rn(-O[j][k], F[k].y, acc.y);
    }
    U[j] = acc;
  }
}

// Green update of one z-pass tile (Algorithm 1 step 5): sm holds the forward
// transformed force F(q) of the tile; the state u(q) is read from and written
// to a.S, and the new u(q) replaces F(q) in sm for the inverse transform.
template <typename T, int CT>
__device__ __forceinline__ void col_green(const ColArgs<T>& a, typename cplx_t<T>::type* sm,
                                          const typename cplx_t<T>::type* ss, size_t base, size_t rstride,
                                          size_t cstride, int x0, int outer, int ncol, int L, int tid, int nthr) {
  const bool c0iso = a.c0iso || a.c0dev != nullptr;
  const T c0a = a.c0dev != nullptr ? a.c0dev[0] : a.c0a;
  const T c0b = a.c0dev != nullptr ? a.c0dev[1] : a.c0b;
  using C = typename cplx_t<T>::type;
  constexpr int W = 3 * CT;
  constexpr int GU = 4;  // points per thread per batch: state loads issued together
  for (int i0 = tid; i0 < L * CT; i0 += GU * nthr) {
    C U[GU][3];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int i = i0 + u * nthr;
      const int z = i / CT, col = i - z * CT;
      if (i < L * CT && col < ncol) {
        if (ss != nullptr) {
#pragma unroll
          for (int c = 0; c < 3; ++c) U[u][c] = ss[z * W + c * CT + col];
        } else {
          const size_t g = base + z * rstride + col;
#pragma unroll
          for (int c = 0; c < 3; ++c) U[u][c] = a.S[c * cstride + g];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int i = i0 + u * nthr;
      const int z = i / CT, col = i - z * CT;
      if (i < L * CT && col < ncol) {
        C F[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) F[c] = sm[z * W + c * CT + col];
        green_apply<T>(a, c0a, c0b, c0iso, x0 + col, outer, z, F, U[u]);
        const size_t g = base + z * rstride + col;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          a.S[c * cstride + g] = U[u][c];
          sm[z * W + c * CT + col] = U[u][c];
        }
      }
    }
  }
}

// col_green for a compile-time length L and block size NT (NT a multiple of CT): thread tid keeps
// column tid % CT and walks z = tid / CT, tid / CT + NT / CT, ..., so exp(-i q_x), its product
// with the block's exp(-i q_y), the state address of its column and whether its (q_x, q_y) can
// be a translation mode are set once; per point only exp(-i q_z) and two products remain.
// tz: a shared-memory copy of the z pass's twiddle table, which holds the z phase factors
// (the same values as tw3).
template <typename T, int CT, int L, int NT>
__device__ __forceinline__ void col_green_fixed(const ColArgs<T>& a, typename cplx_t<T>::type* sm, size_t base,
                                                size_t rstride, size_t cstride, int x0, int outer, int ncol,
                                                int tid, const typename cplx_t<T>::type* tz) {
  using C = typename cplx_t<T>::type;
  static_assert(NT % CT == 0 && (L * CT) % NT == 0, "whole columns per thread");
  constexpr int W = 3 * CT;
  constexpr int ZS = NT / CT;        // z step of a thread
  constexpr int NPT = L * CT / NT;   // points per thread
  // points in groups of GU; the state loads of the next group are issued before the update of
  // the current one (different points), so their latency runs under its arithmetic
  constexpr int GU = NPT < 2 ? NPT : 2;
  static_assert(NPT % GU == 0, "whole groups per thread");
  const int col = tid % CT, zt = tid / CT;
  if (col >= ncol) return;
  const bool c0iso = a.c0iso || a.c0dev != nullptr;
  const T c0a = a.c0dev != nullptr ? a.c0dev[0] : a.c0a;
  const T c0b = a.c0dev != nullptr ? a.c0dev[1] : a.c0b;
  const int h1 = x0 + col, h2 = outer;
  const C ex = __ldg(a.tw1 + h1), ey = __ldg(a.tw2 + h2);
  const C xy = cmul_rn(ex, ey);
  // translation modes q = 0 and (pi, pi, pi): only where (q_x, q_y) is (0, 0) or (pi, pi)
  const int ztrans = (h1 == 0 && h2 == 0) ? 0 : ((2 * h1 == a.n1 && 2 * h2 == a.n2) ? a.n3 / 2 : -1);
  C* Sc = a.S + base + col;
  auto load_group = [&](C (&V)[GU][3], int u0) {
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const size_t g = (size_t)(zt + (u0 + u) * ZS) * rstride;
#pragma unroll
      for (int c = 0; c < 3; ++c) V[u][c] = Sc[c * cstride + g];
    }
  };
  C Un[GU][3];
  load_group(Un, 0);
#pragma unroll
  for (int u0 = 0; u0 < NPT; u0 += GU) {
    C U[GU][3];
#pragma unroll
    for (int u = 0; u < GU; ++u)
#pragma unroll
      for (int c = 0; c < 3; ++c) U[u][c] = Un[u][c];
    if (u0 + GU < NPT) load_group(Un, u0 + GU);
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int z = zt + (u0 + u) * ZS;
      C F[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] = sm[z * W + c * CT + col];
      if (z == ztrans) {
#pragma unroll
        for (int c = 0; c < 3; ++c) U[u][c] = cmk<C>(0, 0);
      } else {
        const C ez = tw_load<true>(tz, z);
        green_core<T>(a, c0a, c0b, c0iso, cmul_rn(ey, ez), xy, cmul_rn(ex, ez), F, U[u]);
      }
      const size_t g = (size_t)z * rstride;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Sc[c * cstride + g] = U[u][c];
        sm[z * W + c * CT + col] = U[u][c];
      }
    }
  }
}

// LF > 0: the transformed length is LF and the block has NT threads, both
// fixed at compile time (hot sizes); LF = 0: both taken at run time; LF = -1:
// run time, plans with a radix-5, 7 or 11 stage.
// TMA (z pass with the state read point by point, fixed lengths): thread 0 loads the tile by
// tensor copies (one per 256 planes) on an mbarrier while every thread issues the state's L2
// prefetch; the wait is bounded (a timeout is recorded in the status).
template <typename T, int CT, int MODE, int LF = 0, int NT = 0, bool TMA = false>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 384 : 768) k_col(const __grid_constant__ ColArgs<T> a_) {
  using C = typename cplx_t<T>::type;
  static_assert(!TMA || (MODE == COL_Z_GREEN && LF > 0), "tensor copies: fixed-length z pass");
  const ColArgs<T> a = col_item_args(a_);
  if (a.st->retired || (a.skip_if_done && a.st->done)) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  // TMA: the tile starts on a 128-byte boundary and its barrier follows it (kColpTmaSlack)
  unsigned char* const smb = TMA ? smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u) : smraw;
  C* sm = reinterpret_cast<C*>(smb);  // [L][3][CT]
  const bool yaxis = (MODE == COL_Y_FWD || MODE == COL_Y_INV);
  const int L = LF > 0 ? LF : (yaxis ? a.n2 : a.n3);
  const int tid = threadIdx.x, nthr = NT > 0 ? NT : (int)blockDim.x;
  const int x0 = blockIdx.x * CT;
  const int outer = blockIdx.y;
  const int ncol = min(CT, a.nh - x0);
  const size_t plane = (size_t)a.n2 * a.P;
  const size_t cstride = (size_t)a.n3 * plane;
  const size_t rstride = yaxis ? (size_t)a.P : plane;
  const size_t base = yaxis ? (size_t)outer * plane + x0 : (size_t)outer * a.P + x0;
  const C* src = (MODE == COL_Z_INV_STATE) ? a.S : a.buf;
  const FftPlan plan = a.plan;
  const C* __restrict__ tw = a.tw;
  constexpr int W = 3 * CT;
  const int ccols = min(CT, a.P - x0);
  // tile load: 16-byte asynchronous copies of the whole tile (every load in
  // flight at once); columns past the row pitch are zero
  constexpr int EPC = 16 / (int)sizeof(C);  // complex values per 16-byte chunk
  constexpr int CPR = CT / EPC;             // chunks per (row, component)
  // fixed lengths: the transforms read their twiddles from the plan's per-stage table in shared
  // memory, 16 bytes behind the tile (and the state tile, when there is one), and the Green step
  // its z phases from a plain copy of the table after it; the host adds 16 + 2 L complex values
  // to the tile's shared memory for them
  C* const tws = reinterpret_cast<C*>(
      smb + (size_t)((MODE == COL_Z_GREEN && a.state_smem) ? 2 : 1) * L * W * sizeof(C) + 16);
  C* const tzs = tws + L;
  auto copy_tables = [&]() {
    if constexpr (LF > 0) {
      stage_twiddles<LF>(tws, tw, tid, nthr);
      if (MODE == COL_Z_GREEN)
        for (int i = tid; i < L; i += nthr) tzs[i] = __ldg(tw + i);
    }
  };
  if constexpr (TMA) {
    uint64_t* const tbar = reinterpret_cast<uint64_t*>(smb + (size_t)L * W * sizeof(C));
    // the copy needs a 128-byte aligned destination and a 64-byte aligned map: checked once,
    // the pass ends with an error status instead of issuing a misaligned copy
    if ((smem_u32(sm) & 127u) != 0 || (reinterpret_cast<uintptr_t>(&a_.tmap) & 63u) != 0) {
      if (tid == 0) a.st->done = DONE_FAULT;
      return;
    }
    if (tid == 0) {
      mbar_init(tbar, 1);
      mbar_init_fence();
      mbar_arrive_expect_tx(tbar, (unsigned)(L * W * sizeof(C)));
#pragma unroll
      for (int h = 0; h < (L + 255) / 256; ++h)
        tma_load_5d(sm + (size_t)h * 256 * W, &a_.tmap, 2 * x0, 0, outer, h * 256, (int)blockIdx.z, tbar);
    }
    for (int i = tid; i < L * 3; i += nthr) {
      const int e = i / 3, c = i - 3 * e;
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.S + c * cstride + base + e * rstride));
    }
    copy_tables();
    __syncthreads();  // the barrier is initialised before anyone waits on it
    if (!mbar_wait(tbar, 0)) {
      if (tid == 0) a.st->done = DONE_TIMEOUT;
    }
  }
  for (int i = tid; !TMA && i < L * 3 * CPR; i += nthr) {
    const int e = i / (3 * CPR), rem = i - e * (3 * CPR), c = rem / CPR, col = (rem - c * CPR) * EPC;
    C* dst = sm + e * W + c * CT + col;
    if (col < ccols) {
      cp_async16(dst, src + c * cstride + base + e * rstride + col);
    } else {
#pragma unroll
      for (int q = 0; q < EPC; ++q) dst[q] = cmk<C>(0, 0);
    }
  }
  cp_async_commit();
  C* ss = nullptr;  // state tile in shared memory (COL_Z_GREEN with state_smem)
  if (TMA) {
    // the tile arrived on the barrier above
  } else if (MODE == COL_Z_GREEN) {
    if (a.state_smem) {
      // the state tile follows the force tile; its copy (a second group) overlaps the forward
      // transform, which waits for the first group only
      ss = sm + (size_t)L * W;
      for (int i = tid; i < L * 3 * CPR; i += nthr) {
        const int e = i / (3 * CPR), rem = i - e * (3 * CPR), c = rem / CPR, col = (rem - c * CPR) * EPC;
        if (col < ccols) cp_async16(ss + e * W + c * CT + col, a.S + c * cstride + base + e * rstride + col);
      }
      cp_async_commit();
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      // the Green step reads the state tile after the forward transform: start
      // moving it into L2 now (one prefetch per 64-byte row segment)
      for (int i = tid; i < L * 3; i += nthr) {
        const int e = i / 3, c = i - 3 * e;
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.S + c * cstride + base + e * rstride));
      }
      cp_async_wait_all();
    }
  } else {
    cp_async_wait_all();
  }
  if (!TMA) copy_tables();
  __syncthreads();
  if constexpr (LF > 0) {
    // compile-time plan; the last stage writes straight to global memory
    ColIO<C> io;
    io.gin = nullptr;
    io.gout = a.buf + base;
    io.cstride = cstride;
    io.rstride = rstride;
    io.ccols = ccols;
    io.ncol = ncol;
    if (MODE == COL_Z_GREEN) {
      fft_col_fixed<LF, W, CT, false, false, false, true>(sm, io, tws, tid, nthr);
      if (ss != nullptr) {
        cp_async_wait_all();
        __syncthreads();
      }
      if constexpr (NT > 0 && NT % CT == 0 && (LF * CT) % NT == 0) {
        if (ss == nullptr) col_green_fixed<T, CT, LF, NT>(a, sm, base, rstride, cstride, x0, outer, ncol, tid, tzs);
        else col_green<T, CT>(a, sm, ss, base, rstride, cstride, x0, outer, ncol, L, tid, nthr);
      } else {
        col_green<T, CT>(a, sm, ss, base, rstride, cstride, x0, outer, ncol, L, tid, nthr);
      }
      __syncthreads();
      fft_col_fixed<LF, W, CT, true, false, true, true>(sm, io, tws, tid, nthr);
    } else {
      fft_col_fixed<LF, W, CT, MODE == COL_Y_INV || MODE == COL_Z_INV_STATE, false, true, true>(sm, io, tws, tid,
                                                                                            nthr);
    }
    return;
  }
  constexpr bool EXT = LF < 0;
  if (MODE == COL_Y_INV || MODE == COL_Z_INV_STATE) {
    fft_smem<true, true, EXT>(sm, 1, W, -1, W, plan.L, plan.nstage, plan.packed, tw, tid, nthr);
  } else {
    fft_smem<false, true, EXT>(sm, 1, W, -1, W, plan.L, plan.nstage, plan.packed, tw, tid, nthr);
  }
  if (MODE == COL_Z_GREEN) {
    if (ss != nullptr) {
      cp_async_wait_all();
      __syncthreads();
    }
    col_green<T, CT>(a, sm, ss, base, rstride, cstride, x0, outer, ncol, L, tid, nthr);
    __syncthreads();
    fft_smem<true, true, EXT>(sm, 1, W, -1, W, plan.L, plan.nstage, plan.packed, tw, tid, nthr);
  }
  for (int i = tid; i < L * W; i += nthr) {
    const int e = i / W, rem = i - e * W, c = rem / CT, col = rem - c * CT;
    if (col < ncol) a.buf[c * cstride + base + e * rstride + col] = sm[i];
  }
}

// Persistent column pass for the compile-time lengths: block j transforms tiles j,
// j + gridDim.x, ... (tile t: x columns (t mod xtiles) * CT, outer index t / xtiles)
// and copies the next tile into its second buffer while it transforms the current
// one, so the copies overlap the arithmetic.  Y_FWD, Y_INV and Z_GREEN (state read
// point by point after an L2 prefetch issued with the tile's copy).
// TMA (y passes): thread 0 issues each tile as tensor copies (one per 256 rows) completing on the
// tile buffer's mbarrier, every thread waits on it (bounded; a timeout is recorded in the status).
template <typename T, int CT, int MODE, int LF, int NT, bool TMA = false>
__global__ void __launch_bounds__(NT, 2) k_colp(const __grid_constant__ ColArgs<T> a_) {
  using C = typename cplx_t<T>::type;
  static_assert(LF > 0 && MODE != COL_Z_INV_STATE, "persistent column pass: fixed lengths, iteration modes");
  static_assert(!TMA || MODE == COL_Y_FWD || MODE == COL_Y_INV || MODE == COL_Z_GREEN, "tensor copies");
  const ColArgs<T> a = col_item_args(a_);
  if (a.st->retired || (a.skip_if_done && a.st->done)) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  constexpr bool yaxis = (MODE == COL_Y_FWD || MODE == COL_Y_INV);
  constexpr int L = LF, W = 3 * CT;
  constexpr int EPC = 16 / (int)sizeof(C);
  constexpr int CPR = CT / EPC;
  // TMA: the tiles start on a 128-byte boundary (tensor copy destinations), the two barriers
  // follow them; the host adds kColpTmaSlack bytes to the dynamic shared memory for this
  unsigned char* const smb = TMA ? smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u) : smraw;
  C* const sm0 = reinterpret_cast<C*>(smb);  // [2][L][3][CT]
  uint64_t* const tbar = reinterpret_cast<uint64_t*>(smb + (size_t)2 * L * W * sizeof(C));
  const int tid = threadIdx.x;
  if (TMA) {
    // the copy needs a 128-byte aligned destination and a 64-byte aligned map: checked once,
    // the pass ends with an error status instead of issuing a misaligned copy
    if ((smem_u32(sm0) & 127u) != 0 || (reinterpret_cast<uintptr_t>(&a_.tmap) & 63u) != 0) {
      if (tid == 0) a.st->done = DONE_FAULT;
      return;
    }
  }
  const size_t plane = (size_t)a.n2 * a.P;
  const size_t cstride = (size_t)a.n3 * plane;
  const size_t rstride = yaxis ? (size_t)a.P : plane;
  const int xtiles = (a.nh + CT - 1) / CT;
  const int ntiles = xtiles * (yaxis ? a.n3 : a.n2);
  // the Green step reads the state tile of tile t after its forward transform: into L2 early
  auto prefetch_state = [&](int t) {
    const int x0 = (t % xtiles) * CT, outer = t / xtiles;
    const size_t base = yaxis ? (size_t)outer * plane + x0 : (size_t)outer * a.P + x0;
    for (int i = tid; i < L * 3; i += NT) {
      const int e = i / 3, c = i - 3 * e;
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.S + c * cstride + base + e * rstride));
    }
  };
  auto load = [&](int t, C* sm) {
    const int x0 = (t % xtiles) * CT, outer = t / xtiles;
    const size_t base = yaxis ? (size_t)outer * plane + x0 : (size_t)outer * a.P + x0;
    const int ccols = min(CT, a.P - x0);
    for (int i = tid; i < L * 3 * CPR; i += NT) {
      const int e = i / (3 * CPR), rem = i - e * (3 * CPR), c = rem / CPR, col = (rem - c * CPR) * EPC;
      C* dst = sm + e * W + c * CT + col;
      if (col < ccols) {
        cp_async16(dst, a.buf + c * cstride + base + e * rstride + col);
      } else {
#pragma unroll
        for (int q = 0; q < EPC; ++q) dst[q] = cmk<C>(0, 0);
      }
    }
    if (MODE == COL_Z_GREEN) prefetch_state(t);
  };
  // tile t into buffer b by tensor copies (thread 0)
  auto load_tma = [&](int t, int b) {
    const int x0 = (t % xtiles) * CT, outer = t / xtiles;
    C* sm = sm0 + (size_t)b * L * W;
    mbar_arrive_expect_tx(&tbar[b], (unsigned)(L * W * sizeof(C)));
#pragma unroll
    for (int h = 0; h < (L + 255) / 256; ++h) {
      if (yaxis) tma_load_5d(sm + (size_t)h * 256 * W, &a_.tmap, 2 * x0, 0, h * 256, outer, (int)blockIdx.z, &tbar[b]);
      else tma_load_5d(sm + (size_t)h * 256 * W, &a_.tmap, 2 * x0, 0, outer, h * 256, (int)blockIdx.z, &tbar[b]);
    }
  };
  // the plan's per-stage twiddle table behind the barriers, then (z pass) a plain copy of the table
  // for the Green step's z phases (read after the first barrier)
  C* const tws = reinterpret_cast<C*>(smb + (size_t)2 * L * W * sizeof(C) + 16);
  C* const tzs = tws + L;
  stage_twiddles<LF>(tws, a.tw, tid, NT);
  if (MODE == COL_Z_GREEN)
    for (int i = tid; i < L; i += NT) tzs[i] = __ldg(a.tw + i);
  bool timed_out = false;
  int t = blockIdx.x;
  if constexpr (TMA) {
    if (tid == 0) {
      mbar_init(&tbar[0], 1);
      mbar_init(&tbar[1], 1);
      mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0 && t < ntiles) load_tma(t, 0);
    if (MODE == COL_Z_GREEN && t < ntiles) prefetch_state(t);
  } else {
    if (t < ntiles) load(t, sm0);
    cp_async_commit();
  }
  for (int k = 0; t < ntiles; ++k, t += gridDim.x) {
    C* sm = sm0 + (size_t)(k & 1) * L * W;
    // the other buffer was freed by the barrier that ended the previous tile
    if constexpr (TMA) {
      if (tid == 0 && t + (int)gridDim.x < ntiles) load_tma(t + gridDim.x, (k + 1) & 1);
      if (MODE == COL_Z_GREEN && t + (int)gridDim.x < ntiles) prefetch_state(t + gridDim.x);
      timed_out |= !mbar_wait(&tbar[k & 1], (unsigned)((k >> 1) & 1));
    } else {
      if (t + (int)gridDim.x < ntiles) load(t + gridDim.x, sm0 + (size_t)((k + 1) & 1) * L * W);
      cp_async_commit();
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    }
    __syncthreads();
    const int x0 = (t % xtiles) * CT, outer = t / xtiles;
    const size_t base = yaxis ? (size_t)outer * plane + x0 : (size_t)outer * a.P + x0;
    ColIO<C> io;
    io.gin = nullptr;
    io.gout = a.buf + base;
    io.cstride = cstride;
    io.rstride = rstride;
    io.ccols = min(CT, a.P - x0);
    io.ncol = min(CT, a.nh - x0);
    if (MODE == COL_Z_GREEN) {
      fft_col_fixed<LF, W, CT, false, false, false, true>(sm, io, tws, tid, NT);
      if constexpr (NT % CT == 0 && (LF * CT) % NT == 0) {
        col_green_fixed<T, CT, LF, NT>(a, sm, base, rstride, cstride, x0, outer, io.ncol, tid, tzs);
      } else {
        col_green<T, CT>(a, sm, nullptr, base, rstride, cstride, x0, outer, io.ncol, L, tid, NT);
      }
      __syncthreads();
      fft_col_fixed<LF, W, CT, true, false, true, true>(sm, io, tws, tid, NT);
    } else {
      fft_col_fixed<LF, W, CT, MODE == COL_Y_INV, false, true, true>(sm, io, tws, tid, NT);
    }
    // this tile's shared writes come before the tensor copy that refills the buffer
    if (TMA) fence_async_smem();
    __syncthreads();
  }
  cp_async_wait_all();
  if (TMA && timed_out) a.st->done = DONE_TIMEOUT;
}

}  // namespace hs
