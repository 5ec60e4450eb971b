// Real-space pass of the tetrahedral-stencil basic scheme, marching along z.
//
// One block owns a tile of TY corner rows (y) of one z-chunk and all N1 x
// positions (thread x <-> column x).  For every voxel plane p it
//   1. brings the corner plane p (rows y0-1 .. y0+TY) into shared memory:
//      either by an inverse real FFT along x of the y/z-transformed state
//      (two real rows packed in one complex sequence), or (REAL = true) by
//      plain loads of a real FP64 displacement field;
//   2. computes, per voxel, the T1 and T2 strains of the two inscribed
//      tetrahedra (Eqs. deps, DA1-DA2; T1 = corners whose offset signs
//      multiply to +1, T2 = the centrally symmetric set), the stresses
//      sigma^T = lambda(r) : (E + deps^T) (Algorithm 1 step 3) and
//   3. scatters the adjoint stencil: the nodal force
//      F_k(c) = dE/du_k(c) = 1/2 sum_T sum_{voxels r of c} 1/2 s_i sigma^T_ik(r)
//      (the real-space form of Eq. der_E_dep_Q) into per-thread accumulators
//      for corner planes p-1 and p; contributions to column x-1 go left by
//      warp shuffle (lane 0's through shared memory);
//   4. when corner plane p-1 is complete: forward real FFT along x (packed
//      pairs) and store (FORCE), or store the real force (REAL FORCE).
// FIELDS writes eps = E + 1/2(deps^T1 + deps^T2) and sigma = 1/2(sigma^T1 +
// sigma^T2) (Eq. final_fields) instead; EMIT adds the inverse-transformed
// displacement into an FP64 real field.
//
// Sums of sigma^T1, sigma^T2 and |F|^2 go through reduce_and_finalize(),
// which evaluates the stopping test of Eqs. (L2-norm, tolerance).
#pragma once
#include "common.cuh"

namespace hs {

enum { MODE_FORCE = 0, MODE_FIELDS = 1, MODE_EMIT = 2 };

template <typename T> struct MarchArgs {
  using C = typename cplx_t<T>::type;
  const C* in;           // y/z-transformed displacement, [3][n3][n2][P]
  C* out;                // x-transformed force, [3][n3][n2][P]
  const uint16_t* ids;   // phase id per voxel [n3][n2][n1]
  const T* mat;          // phase table (MatIso / MatAniso layout)
  T E[6];                // macroscopic strain, tensor components, Voigt order
  const C* tw1;          // w_N1^j, j < N1
  FftPlan plan1;
  int n1, n2, n3, P, zc;
  double* partials;
  DevStatus* st;
  double* hist;
  const float* src;      // optional real force added to F, [3][n3][n2][n1]
  void* eps_out;         // FIELDS: [6][n3][n2][n1]
  void* sig_out;
  int out_f32;
  double* u64;           // EMIT: += u ; REAL: input displacement [3][n3][n2][n1]
  float* fout;           // REAL FORCE: real force [3][n3][n2][n1]
  int skip_if_done;
};

// corner values u[ox][oy][oz][comp]; offset index 1 means coordinate - 1
template <typename T>
__device__ __forceinline__ void tetra_strains(const T (&u)[2][2][2][3], const T* E, T* e1, T* e2) {
  T g1[3][3], g2[3][3];  // g[i][j] = D_i u_j
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    // T1: corners (0,0,0), (0,-1,-1), (-1,-1,0), (-1,0,-1)
    const T a = u[0][0][0][j], b = u[0][1][1][j], c = u[1][1][0][j], d = u[1][0][1][j];
    const T p = a + b, q = c + d, m = a - b, n = c - d;
    g1[0][j] = T(0.5) * (p - q);
    g1[1][j] = T(0.5) * (m - n);
    g1[2][j] = T(0.5) * (m + n);
    // T2: corners (0,-1,0), (0,0,-1), (-1,-1,-1), (-1,0,0)
    const T a2 = u[0][1][0][j], b2 = u[0][0][1][j], c2 = u[1][1][1][j], d2 = u[1][0][0][j];
    const T p2 = a2 + b2, q2 = c2 + d2, m2 = b2 - a2, n2 = d2 - c2;
    g2[0][j] = T(0.5) * (p2 - q2);
    g2[1][j] = T(0.5) * (m2 + n2);
    g2[2][j] = T(0.5) * (n2 - m2);
  }
  e1[0] = E[0] + g1[0][0];
  e1[1] = E[1] + g1[1][1];
  e1[2] = E[2] + g1[2][2];
  e1[3] = E[3] + E[3] + g1[1][2] + g1[2][1];
  e1[4] = E[4] + E[4] + g1[0][2] + g1[2][0];
  e1[5] = E[5] + E[5] + g1[0][1] + g1[1][0];
  e2[0] = E[0] + g2[0][0];
  e2[1] = E[1] + g2[1][1];
  e2[2] = E[2] + g2[2][2];
  e2[3] = E[3] + E[3] + g2[1][2] + g2[2][1];
  e2[4] = E[4] + E[4] + g2[0][2] + g2[2][0];
  e2[5] = E[5] + E[5] + g2[0][1] + g2[1][0];
}

// Corner plane zz (rows y0-1 .. y0+TY) into shared memory (see file comment).
// Engineering strain of one tetrahedron (tt = 0: T1, tt = 1: T2).
template <typename T>
__device__ __forceinline__ void tetra_strain_one(const T (&u)[2][2][2][3], const T* E, int tt, T* e) {
  T g[3][3];  // g[i][j] = D_i u_j
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (tt == 0) {
      const T a = u[0][0][0][j], b = u[0][1][1][j], c = u[1][1][0][j], d = u[1][0][1][j];
      const T p = a + b, q = c + d, m = a - b, n = c - d;
      g[0][j] = T(0.5) * (p - q);
      g[1][j] = T(0.5) * (m - n);
      g[2][j] = T(0.5) * (m + n);
    } else {
      const T a = u[0][1][0][j], b = u[0][0][1][j], c = u[1][1][1][j], d = u[1][0][0][j];
      const T p = a + b, q = c + d, m = b - a, n = d - c;
      g[0][j] = T(0.5) * (p - q);
      g[1][j] = T(0.5) * (m + n);
      g[2][j] = T(0.5) * (n - m);
    }
  }
  e[0] = E[0] + g[0][0];
  e[1] = E[1] + g[1][1];
  e[2] = E[2] + g[2][2];
  e[3] = E[3] + E[3] + g[1][2] + g[2][1];
  e[4] = E[4] + E[4] + g[0][2] + g[2][0];
  e[5] = E[5] + E[5] + g[0][1] + g[1][0];
}

template <typename T, int TY, bool REAL>
__device__ __forceinline__ void march_load_plane(
    typename cplx_t<T>::type* __restrict__ ring, T* __restrict__ rring, int slot, int zz,
    const typename cplx_t<T>::type* __restrict__ in, const double* __restrict__ u64, int n1, int n2, int n3,
    int P, int y0, const FftPlan& plan, const typename cplx_t<T>::type* __restrict__ tw1, int tid, int nthr) {
  using C = typename cplx_t<T>::type;
  constexpr int NR = TY + 2;
  constexpr int NSI = 3 * NR / 2;
  zz = ((zz % n3) + n3) % n3;
  const size_t plane_stride = (size_t)n2 * P;
  const size_t comp_stride = (size_t)n3 * plane_stride;
  const size_t rplane = (size_t)n2 * n1;
  const size_t rcomp = (size_t)n3 * rplane;
  if (REAL) {
    for (int i = tid; i < 3 * NR * n1; i += nthr) {
      const int r = i / n1, k = i - r * n1;
      const int c = r / NR, j = r - c * NR;
      const int yy = (y0 - 1 + j + n2) % n2;
      rring[slot * 3 * NR * n1 + i] = (T)u64[c * rcomp + (size_t)zz * rplane + (size_t)yy * n1 + k];
    }
    __syncthreads();
  } else {
    C* R = ring + slot * NSI * n1;
    const int half = n1 / 2;
    for (int i = tid; i < NSI * n1; i += nthr) {
      const int q = i / n1, k = i - q * n1;
      const int ra = 2 * q;
      const int c = ra / NR, ja = ra - c * NR;
      const int ya = (y0 - 1 + ja + n2) % n2, yb = (y0 + ja + n2) % n2;
      const int kk = (k <= half) ? k : n1 - k;
      const size_t base = c * comp_stride + (size_t)zz * plane_stride + kk;
      C A = in[base + (size_t)ya * P];
      C B = in[base + (size_t)yb * P];
      if (kk == 0 || kk == half) { A.y = 0; B.y = 0; }
      C Z;
      if (k <= half) { Z.x = A.x - B.y; Z.y = A.y + B.x; }
      else { Z.x = A.x + B.y; Z.y = B.x - A.y; }
      R[i] = Z;
    }
    __syncthreads();
    HS_FFT(true, R, n1, 1, NSI, plan, tw1, tid, nthr);
  }
}

template <typename T, int TY, bool REAL>
__device__ __forceinline__ T march_u(const typename cplx_t<T>::type* __restrict__ ring,
                                     const T* __restrict__ rring, int slot, int c, int j, int xx, int n1) {
  constexpr int NR = TY + 2;
  constexpr int NSI = 3 * NR / 2;
  if (REAL) return rring[((slot * 3 + c) * NR + j) * n1 + xx];
  const int r = c * NR + j;
  const auto z = ring[(slot * NSI + (r >> 1)) * n1 + xx];
  return (r & 1) ? z.y : z.x;
}

template <typename T, int TY, class MAT, int MODE, bool REAL>
__global__ void __launch_bounds__(512) k_march(const MarchArgs<T> a, const MAT mat) {
  using C = typename cplx_t<T>::type;
  constexpr int NR = TY + 2;          // corner rows per plane (1 halo row each side)
  constexpr int NSI = 3 * NR / 2;     // packed complex sequences per plane
  constexpr int NSF = 3 * TY / 2;     // packed sequences of the output force
  if (a.skip_if_done && a.st->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3, P = a.P, nh = n1 / 2 + 1;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const int y0 = blockIdx.x * TY;
  const int z0 = blockIdx.y * a.zc;
  const int zc = min(a.zc, n3 - z0);
  const size_t plane_stride = (size_t)n2 * P;   // complex elements per (comp, z)
  const size_t comp_stride = (size_t)n3 * plane_stride;
  const size_t rplane = (size_t)n2 * n1;        // real elements per z plane
  const size_t rcomp = (size_t)n3 * rplane;
  const C* __restrict__ in = a.in;
  C* __restrict__ out = a.out;
  const uint16_t* __restrict__ ids = a.ids;
  const C* __restrict__ tw1 = a.tw1;
  const FftPlan plan = a.plan1;

  // shared memory carve
  C* ring = reinterpret_cast<C*>(smraw);                           // [2][NSI][n1] (complex path)
  T* rring = reinterpret_cast<T*>(smraw);                          // [2][3][NR][n1] (REAL path)
  const size_t ring_bytes = REAL ? sizeof(T) * 2 * 3 * NR * n1 : sizeof(C) * 2 * NSI * n1;
  C* fbuf = reinterpret_cast<C*>(smraw + ring_bytes);              // [NSF][n1]
  const size_t fbuf_bytes = (REAL || MODE != MODE_FORCE) ? 0 : sizeof(C) * NSF * n1;
  T* edge = reinterpret_cast<T*>(smraw + ring_bytes + fbuf_bytes); // [nwarps][TY+1][12]
  double* red = reinterpret_cast<double*>(smraw + ring_bytes + fbuf_bytes +
                                          ((sizeof(T) * nwarps * (TY + 1) * 12 + 15) & ~size_t(15)));

  const int x = tid;
  const bool xact = x < n1;
  const int xm = (x == 0) ? n1 - 1 : x - 1;
  const int xr = xact ? x : 0, xmr = xact ? xm : 0;

  if (MODE == MODE_EMIT) {
    double* __restrict__ u64 = a.u64;
    for (int p = z0; p < z0 + zc; ++p) {
      march_load_plane<T, TY, false>(ring, rring, 0, p, in, nullptr, n1, n2, n3, P, y0, plan, tw1, tid, nthr);
      if (xact) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < TY; ++r)
            u64[c * rcomp + (size_t)p * rplane + (size_t)(y0 + r) * n1 + x] +=
                (double)march_u<T, TY, false>(ring, rring, 0, c, r + 1, x, n1);
      }
      __syncthreads();
    }
    return;
  }

  T Fp[TY][3], Fn[TY][3];
#pragma unroll
  for (int r = 0; r < TY; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) { Fp[r][k] = 0; Fn[r][k] = 0; }
  T sacc[6];  // sum over owned voxels of sigma^T1 + sigma^T2
#pragma unroll
  for (int i = 0; i < 6; ++i) sacc[i] = 0;
  T facc = 0;
  T E[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) E[i] = a.E[i];

  const bool recv_shfl = (lane < 31) && (x + 1 < n1);
  const bool recv_edge = xact && !recv_shfl;
  const int src_warp = ((x + 1) % n1) >> 5;

  march_load_plane<T, TY, REAL>(ring, rring, 0, z0 - 1, in, a.u64, n1, n2, n3, P, y0, plan, tw1, tid, nthr);
  const int pend = (MODE == MODE_FORCE) ? z0 + zc : z0 + zc - 1;
  for (int p = z0; p <= pend; ++p) {
    const int sc = (p - z0 + 1) & 1, sp = sc ^ 1;
    march_load_plane<T, TY, REAL>(ring, rring, sc, p, in, a.u64, n1, n2, n3, P, y0, plan, tw1, tid, nthr);
    const int pz = p % n3;
    const bool own_plane = p < z0 + zc;

    // ---- per-voxel work: rows jj = 1..TY+1 (voxel y = y0 + jj - 1) ----
    T uc[2][3][2];  // cached corner values of row jj: [ox][comp][oz]
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uc[0][c][0] = march_u<T, TY, REAL>(ring, rring, sc, c, 0, xr, n1);
      uc[0][c][1] = march_u<T, TY, REAL>(ring, rring, sp, c, 0, xr, n1);
      uc[1][c][0] = march_u<T, TY, REAL>(ring, rring, sc, c, 0, xmr, n1);
      uc[1][c][1] = march_u<T, TY, REAL>(ring, rring, sp, c, 0, xmr, n1);
    }
#pragma unroll
    for (int jj = 1; jj <= TY + 1; ++jj) {
      if (MODE == MODE_FIELDS && jj == TY + 1) break;
      T u[2][2][2][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
          u[ox][1][0][c] = uc[ox][c][0];
          u[ox][1][1][c] = uc[ox][c][1];
        }
        const T v00 = march_u<T, TY, REAL>(ring, rring, sc, c, jj, xr, n1);
        const T v01 = march_u<T, TY, REAL>(ring, rring, sp, c, jj, xr, n1);
        const T v10 = march_u<T, TY, REAL>(ring, rring, sc, c, jj, xmr, n1);
        const T v11 = march_u<T, TY, REAL>(ring, rring, sp, c, jj, xmr, n1);
        u[0][0][0][c] = v00; u[0][0][1][c] = v01; u[1][0][0][c] = v10; u[1][0][1][c] = v11;
        uc[0][c][0] = v00; uc[0][c][1] = v01; uc[1][c][0] = v10; uc[1][c][1] = v11;
      }
      const int yv = (y0 + jj - 1) % n2;
      const int ph = __ldg(ids + ((size_t)pz * n2 + yv) * n1 + xr);
      if (MODE == MODE_FIELDS) {
        T e1[6], e2[6], s1[6], s2[6];
        tetra_strains(u, E, e1, e2);
        mat.stress(ph, e1, s1);
        mat.stress(ph, e2, s2);
        if (xact && own_plane) {
          const size_t o = (size_t)pz * rplane + (size_t)yv * n1 + x;
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            const T ev = T(0.5) * (e1[i] + e2[i]) * (i < 3 ? T(1) : T(0.5));
            const T sv = T(0.5) * (s1[i] + s2[i]);
            if (a.out_f32) {
              reinterpret_cast<float*>(a.eps_out)[i * rcomp + o] = (float)ev;
              reinterpret_cast<float*>(a.sig_out)[i * rcomp + o] = (float)sv;
            } else {
              reinterpret_cast<double*>(a.eps_out)[i * rcomp + o] = (double)ev;
              reinterpret_cast<double*>(a.sig_out)[i * rcomp + o] = (double)sv;
            }
          }
        }
        continue;
      }
      const bool acc_sig = xact && own_plane && jj <= TY;
      // ---- T1, then T2: strain, stress, adjoint stencil ----
#pragma unroll
      for (int tt = 0; tt < 2; ++tt) {
        T ev[6], sv[6];
        tetra_strain_one(u, E, tt, ev);
        mat.stress(ph, ev, sv);
        if (!xact) {
#pragma unroll
          for (int i = 0; i < 6; ++i) sv[i] = 0;
        }
        if (acc_sig) {
#pragma unroll
          for (int i = 0; i < 6; ++i) sacc[i] += sv[i];
        }
        // per force component k: (sigma_1k, sigma_2k, sigma_3k)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int i1 = (k == 0) ? 0 : (k == 1 ? 5 : 4);
          const int i2 = (k == 0) ? 5 : (k == 1 ? 1 : 3);
          const int i3 = (k == 0) ? 4 : (k == 1 ? 3 : 2);
          const T Ps = sv[i1] + sv[i2], Ms = sv[i1] - sv[i2], Zs = sv[i3];
          const T q = T(0.25);
          T l0, l1;  // left-going: T1: a3 -> Fn[jj-2], a4 -> Fp[jj-1]; T2: a1 -> Fp[jj-2], a2 -> Fn[jj-1]
          if (tt == 0) {
            if (jj - 1 < TY) Fn[jj - 1][k] += q * (Ps + Zs);        // T1 a1 (0,0,0)
            if (jj - 2 >= 0) Fp[jj - 2][k] += q * (Ms - Zs);        // T1 a2 (0,-1,-1)
            l0 = q * (Zs - Ps);                                     // T1 a3 (-1,-1,0)
            l1 = -q * (Ms + Zs);                                    // T1 a4 (-1,0,-1)
          } else {
            if (jj - 2 >= 0) Fn[jj - 2][k] += q * (Ms + Zs);        // T2 a3 (0,-1,0)
            if (jj - 1 < TY) Fp[jj - 1][k] += q * (Ps - Zs);        // T2 a4 (0,0,-1)
            l0 = -q * (Ps + Zs);                                    // T2 a1 (-1,-1,-1)
            l1 = q * (Zs - Ms);                                     // T2 a2 (-1,0,0)
          }
          const T g0 = __shfl_down_sync(0xffffffffu, l0, 1);
          const T g1 = __shfl_down_sync(0xffffffffu, l1, 1);
          if (lane == 0) {
            edge[(warp * (TY + 1) + (jj - 1)) * 12 + (2 * tt) * 3 + k] = l0;
            edge[(warp * (TY + 1) + (jj - 1)) * 12 + (2 * tt + 1) * 3 + k] = l1;
          }
          if (recv_shfl) {
            if (tt == 0) {
              if (jj - 2 >= 0) Fn[jj - 2][k] += g0;
              if (jj - 1 < TY) Fp[jj - 1][k] += g1;
            } else {
              if (jj - 2 >= 0) Fp[jj - 2][k] += g0;
              if (jj - 1 < TY) Fn[jj - 1][k] += g1;
            }
          }
        }
      }
    }
    if (MODE == MODE_FIELDS) {
      __syncthreads();
      continue;
    }
    __syncthreads();
    if (recv_edge) {
#pragma unroll
      for (int jj = 1; jj <= TY + 1; ++jj)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T* e = edge + (src_warp * (TY + 1) + (jj - 1)) * 12;
          if (jj - 2 >= 0) Fn[jj - 2][k] += e[0 * 3 + k];
          if (jj - 1 < TY) Fp[jj - 1][k] += e[1 * 3 + k];
          if (jj - 2 >= 0) Fp[jj - 2][k] += e[2 * 3 + k];
          if (jj - 1 < TY) Fn[jj - 1][k] += e[3 * 3 + k];
        }
    }
    if (p > z0) {
      // corner plane p-1 is complete
      const int zp = (p - 1) % n3;
      if (a.src != nullptr && xact) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < TY; ++r)
            Fp[r][c] += (T)a.src[c * rcomp + (size_t)zp * rplane + (size_t)(y0 + r) * n1 + x];
      }
      if (xact) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < TY; ++r) facc += Fp[r][c] * Fp[r][c];
      }
      if (REAL) {
        if (xact && a.fout != nullptr) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < TY; ++r)
              a.fout[c * rcomp + (size_t)zp * rplane + (size_t)(y0 + r) * n1 + x] = (float)Fp[r][c];
        }
      } else {
        if (xact) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < TY; r += 2) {
              C z;
              z.x = Fp[r][c];
              z.y = Fp[r + 1][c];
              fbuf[((c * TY + r) >> 1) * n1 + x] = z;
            }
        }
        __syncthreads();
        HS_FFT(false, fbuf, n1, 1, NSF, plan, tw1, tid, nthr);
        for (int i = tid; i < NSF * nh; i += nthr) {
          const int q = i / nh, k = i - q * nh;
          const C Zk = fbuf[q * n1 + k];
          const C Zn = fbuf[q * n1 + (k == 0 ? 0 : n1 - k)];
          C A, B;
          A.x = T(0.5) * (Zk.x + Zn.x);
          A.y = T(0.5) * (Zk.y - Zn.y);
          B.x = T(0.5) * (Zk.y + Zn.y);
          B.y = T(0.5) * (Zn.x - Zk.x);
          const int ra = 2 * q;
          const int c = ra / TY, r = ra - c * TY;
          const size_t o = c * comp_stride + (size_t)zp * plane_stride + (size_t)(y0 + r) * P + k;
          out[o] = A;
          out[o + P] = B;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < TY; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) { Fp[r][k] = Fn[r][k]; Fn[r][k] = 0; }
  }
  if (MODE != MODE_FORCE) return;
  double acc[NRED];
#pragma unroll
  for (int i = 0; i < 6; ++i) acc[i] = (double)sacc[i];
  acc[6] = (double)facc;
  reduce_and_finalize(acc, a.partials, a.st, a.hist, red);
}

}  // namespace hs
