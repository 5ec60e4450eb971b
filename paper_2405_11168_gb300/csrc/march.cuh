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

// MODE_FORCE_FIELDS: MODE_FORCE that also writes the fields of MODE_FIELDS (the
// last FP64 residual sweep of a refined solve)
enum { MODE_FORCE = 0, MODE_FIELDS = 1, MODE_EMIT = 2, MODE_FORCE_FIELDS = 3 };

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
  double* u64;           // EMIT: += u
  const T* ureal;        // REAL: input displacement [3][n3][n2][n1]
  void* fout;            // REAL FORCE: real force [3][n3][n2][n1], float if fout_f32 else T
  int fout_f32;
  int skip_if_done;
  const double* Edev;    // not null: the macroscopic strain is read here (applied-stress control)
  const T* sig0;         // not null: lambda(ph) : eps0(ph) per phase, Voigt [nphase][6] (eigenstrain)
  size_t zstride;        // batched launches: bytes between the workspaces of consecutive items
                         // (eps_out and sig_out do not move: batched launches write no fields)
};

// The arguments of item blockIdx.z of a batched launch (every workspace pointer moved).
template <typename T> __device__ __forceinline__ MarchArgs<T> march_item_args(const MarchArgs<T>& a) {
  if (a.zstride == 0) return a;
  MarchArgs<T> b = a;
  const size_t o = (size_t)blockIdx.z * a.zstride;
  b.in = zshift(a.in, o);
  b.out = zshift(a.out, o);
  b.ids = zshift(a.ids, o);
  b.mat = zshift(a.mat, o);
  b.tw1 = zshift(a.tw1, o);
  b.partials = zshift(a.partials, o);
  b.st = zshift(a.st, o);
  b.hist = zshift(a.hist, o);
  b.src = zshift(a.src, o);
  b.u64 = zshift(a.u64, o);
  b.ureal = zshift(a.ureal, o);
  b.fout = zshift(a.fout, o);
  b.Edev = zshift(a.Edev, o);
  b.sig0 = zshift(a.sig0, o);
  return b;
}

// Macroscopic strain of this evaluation: the kernel parameter, or the device
// copy that the applied-stress loop updates.
template <typename T> __device__ __forceinline__ T macro_E(const MarchArgs<T>& a, int i) {
  return a.Edev != nullptr ? (T)a.Edev[i] : a.E[i];
}

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

// Engineering strain E + deps of one tetrahedron (tt = 0: T1, tt = 1: T2) from
// the unscaled differences 2 D_i u_j, the factor 1/2 folded into one FMA.
template <typename T>
__device__ __forceinline__ void tetra_strain_fast(const T (&u)[2][2][2][3], const T* E, int tt, T* e) {
  T g[3][3];  // g[i][j] = 2 D_i u_j
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (tt == 0) {
      const T a = u[0][0][0][j], b = u[0][1][1][j], c = u[1][1][0][j], d = u[1][0][1][j];
      const T p = a + b, q = c + d, m = a - b, n = c - d;
      g[0][j] = p - q;
      g[1][j] = m - n;
      g[2][j] = m + n;
    } else {
      const T a = u[0][1][0][j], b = u[0][0][1][j], c = u[1][1][1][j], d = u[1][0][0][j];
      const T p = a + b, q = c + d, m = b - a, n = d - c;
      g[0][j] = p - q;
      g[1][j] = m + n;
      g[2][j] = n - m;
    }
  }
  const T h = T(0.5);
  e[0] = fma(h, g[0][0], E[0]);
  e[1] = fma(h, g[1][1], E[1]);
  e[2] = fma(h, g[2][2], E[2]);
  e[3] = fma(h, g[1][2] + g[2][1], E[3] + E[3]);
  e[4] = fma(h, g[0][2] + g[2][0], E[4] + E[4]);
  e[5] = fma(h, g[0][1] + g[1][0], E[5] + E[5]);
}

// Shared-memory layout of k_march (host and device use the same function).
struct MarchLayout {
  size_t ring, fbuf, stage, ids, src, edge, red, bar, total;
  int n1i, n1s;  // row pitches (elements) of the ids and source stages
};

__host__ __device__ inline size_t hs_align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline MarchLayout march_layout(int n1, int P, int nthr, int ty, int mode, bool real,
                                                    bool has_src, int tsize) {
  MarchLayout L;
  const int NR = ty + 2, NSI = 3 * NR / 2, NSF = 3 * ty / 2;
  const size_t cs = 2 * (size_t)tsize;
  L.n1i = (n1 + 7) & ~7;
  L.n1s = (n1 + 3) & ~3;
  size_t off = 0;
  L.ring = off;
  off += hs_align16(real ? (size_t)tsize * 3 * 3 * NR * n1 : cs * 2 * NSI * rpitch(n1));
  L.fbuf = off;
  off += hs_align16((real || mode != MODE_FORCE) ? 0 : cs * NSF * rpitch(n1));
  L.stage = off;
  off += hs_align16(real ? 0 : cs * 3 * NR * (size_t)P);
  L.ids = off;
  off += hs_align16(mode == MODE_EMIT ? 0 : (size_t)2 * 2 * (ty + 1) * L.n1i);
  L.src = off;
  off += hs_align16(has_src ? (size_t)4 * 2 * 3 * ty * L.n1s : 0);
  L.edge = off;
  off += hs_align16((size_t)tsize * (nthr / 32) * (ty + 1) * 12);
  L.red = off;
  off += 32 * NRED * 8;
  L.bar = off;  // three mbarriers (bulk plane copies of the FP32 real-space pass)
  off += 32;
  L.total = off;
  return L;
}

template <typename T> struct MarchPtrs {
  const typename cplx_t<T>::type* in;
  const T* ureal;
  const uint16_t* ids;
  const float* src;
  typename cplx_t<T>::type* stage;
  T* rring;
  uint16_t* sids;
  float* ssrc;
  int n1, n2, n3, P, y0, n1i, n1s;
};

// Asynchronous prefetch of one plane's inputs: u rows of corner plane pu
// (complex: into the staging rows; REAL: into ring slot rslot), ids rows of
// voxel plane pu into ids buffer ib, source rows of output plane ps into
// source buffer ib (ps < 0: none).  Ends with a commit of the copy group.
template <typename T, int TY, bool REAL>
__device__ __forceinline__ void march_prefetch(const MarchPtrs<T>& m, int tid, int nthr, int pu, int rslot, int ib,
                                               int ps, bool want_ids) {
  using C = typename cplx_t<T>::type;
  constexpr int NR = TY + 2;
  constexpr int EPC = 16 / (int)sizeof(C);
  const int n1 = m.n1, n2 = m.n2, n3 = m.n3, P = m.P, y0 = m.y0;
  const size_t rplane = (size_t)n2 * n1, rcomp = (size_t)n3 * rplane;
  const size_t plane_stride = (size_t)n2 * P, comp_stride = (size_t)n3 * plane_stride;
  const int gz = ((pu % n3) + n3) % n3;
  if (REAL) {
    constexpr int EPR = 16 / (int)sizeof(T);  // real values per 16-byte chunk
    T* dst0 = m.rring + (size_t)rslot * 3 * NR * n1;
    if (n1 % EPR == 0) {
      const int nch = n1 / EPR;
      for (int i = tid; i < 3 * NR * nch; i += nthr) {
        const int r = i / nch, ch = i - r * nch;
        const int c = r / NR, j = r - c * NR;
        const int gy = (y0 - 1 + j + n2) % n2;
        cp_async16(dst0 + (size_t)r * n1 + EPR * ch,
                   m.ureal + c * rcomp + (size_t)gz * rplane + (size_t)gy * n1 + EPR * ch);
      }
    } else if (tid < n1) {
      for (int r = 0; r < 3 * NR; ++r) {
        const int c = r / NR, j = r - c * NR;
        const int gy = (y0 - 1 + j + n2) % n2;
        dst0[(size_t)r * n1 + tid] = m.ureal[c * rcomp + (size_t)gz * rplane + (size_t)gy * n1 + tid];
      }
    }
  } else {
    const int nh = n1 / 2 + 1;
    const int nch = (nh + EPC - 1) / EPC;
    for (int i = tid; i < 3 * NR * nch; i += nthr) {
      const int r = i / nch, ch = i - r * nch;
      const int c = r / NR, j = r - c * NR;
      const int gy = (y0 - 1 + j + n2) % n2;
      cp_async16(m.stage + (size_t)r * P + ch * EPC,
                 m.in + c * comp_stride + (size_t)gz * plane_stride + (size_t)gy * P + ch * EPC);
    }
  }
  if (want_ids) {
    uint16_t* d = m.sids + (size_t)ib * (TY + 1) * m.n1i;
    if ((n1 & 7) == 0) {
      const int nch = n1 / 8;
      for (int i = tid; i < (TY + 1) * nch; i += nthr) {
        const int r = i / nch, ch = i - r * nch;
        const int gy = (y0 + r) % n2;
        cp_async16(d + (size_t)r * m.n1i + 8 * ch, m.ids + ((size_t)gz * n2 + gy) * n1 + 8 * ch);
      }
    } else if (tid < n1) {
      for (int r = 0; r <= TY; ++r) d[(size_t)r * m.n1i + tid] = m.ids[((size_t)gz * n2 + (y0 + r) % n2) * n1 + tid];
    }
  }
  if (m.src != nullptr && ps >= 0) {
    float* d = m.ssrc + (size_t)ib * 3 * TY * m.n1s;
    const int zs = ps % n3;
    if ((n1 & 3) == 0) {
      const int nch = n1 / 4;
      for (int i = tid; i < 3 * TY * nch; i += nthr) {
        const int r = i / nch, ch = i - r * nch;
        const int c = r / TY, rr = r - c * TY;
        cp_async16(d + (size_t)r * m.n1s + 4 * ch, m.src + c * rcomp + (size_t)zs * rplane + (size_t)(y0 + rr) * n1 + 4 * ch);
      }
    } else if (tid < n1) {
      for (int r = 0; r < 3 * TY; ++r) {
        const int c = r / TY, rr = r - c * TY;
        d[(size_t)r * m.n1s + tid] = m.src[c * rcomp + (size_t)zs * rplane + (size_t)(y0 + rr) * n1 + tid];
      }
    }
  }
  cp_async_commit();
}

// Staged raw rows -> packed complex sequences of ring slot `slot` (two real
// rows per sequence: Z = A + iB with the Hermitian extension of the half
// spectra; imaginary parts of the k = 0 and k = N1/2 bins dropped).
template <typename T, int TY>
__device__ __forceinline__ void march_pack(const MarchPtrs<T>& m, typename cplx_t<T>::type* ring, int x, bool xact,
                                           int slot) {
  using C = typename cplx_t<T>::type;
  constexpr int NSI = 3 * (TY + 2) / 2;
  const int n1 = m.n1, P = m.P;
  const int n1p = rpitch(n1);
  C* R = ring + slot * NSI * n1p;
  const int half = n1 / 2;
  if (xact) {
    const int k = x;
    const int kk = (k <= half) ? k : n1 - k;
#pragma unroll
    for (int q = 0; q < NSI; ++q) {
      C A = m.stage[(size_t)(2 * q) * P + kk];
      C B = m.stage[(size_t)(2 * q + 1) * P + kk];
      if (kk == 0 || kk == half) { A.y = 0; B.y = 0; }
      C Z;
      if (k <= half) { Z.x = A.x - B.y; Z.y = A.y + B.x; }
      else { Z.x = A.x + B.y; Z.y = B.x - A.y; }
      R[q * n1p + rpad(k)] = Z;
    }
  }
  __syncthreads();
}

template <typename T, int TY, bool REAL>
__device__ __forceinline__ T march_u(const typename cplx_t<T>::type* ring, const T* rring, int n1, int slot, int c,
                                     int j, int xx) {
  constexpr int NR = TY + 2;
  constexpr int NSI = 3 * NR / 2;
  if (REAL) return rring[((size_t)slot * 3 * NR + c * NR + j) * n1 + xx];
  const int r = c * NR + j;
  const auto z = ring[(slot * NSI + (r >> 1)) * rpitch(n1) + rpad(xx)];
  return (r & 1) ? z.y : z.x;
}

// BATCH: a batched launch (grid.z items, every workspace pointer moved per item); a single
// solve's launch uses the arguments as they come.
// Blocks of up to 512 threads; the FP64 tile of 8 rows takes blocks of at most 256 (N1 <= 256), so
// that its registers (up to 255) hold the FP64 sweep without spills.
template <typename T, int TY, class MAT, int MODE, bool REAL, bool BATCH = false>
__global__ void __launch_bounds__((sizeof(T) == 8 && TY == 8) ? 256 : 512) k_march(const MarchArgs<T> a_,
                                                                                    const MAT mat_) {
  using C = typename cplx_t<T>::type;
  constexpr int NR = TY + 2;          // corner rows per plane (1 halo row each side)
  constexpr int NSI = 3 * NR / 2;     // packed complex sequences per plane
  constexpr int NSF = 3 * TY / 2;     // packed sequences of the output force
  constexpr int EPC = 16 / (int)sizeof(C);
  const MarchArgs<T> a = BATCH ? march_item_args(a_) : a_;
  MAT mat = mat_;
  if (BATCH) mat.tab = a.mat;
  if (a.st->retired || (a.skip_if_done && a.st->done)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3, P = a.P, nh = n1 / 2 + 1;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
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
  const bool has_src = (a.src != nullptr);

  const MarchLayout lay = march_layout(n1, P, nthr, TY, MODE, REAL, has_src, (int)sizeof(T));
  C* ring = reinterpret_cast<C*>(smraw + lay.ring);      // complex: [2][NSI][n1]
  T* rring = reinterpret_cast<T*>(smraw + lay.ring);     // REAL: [3][3*NR][n1]
  C* fbuf = reinterpret_cast<C*>(smraw + lay.fbuf);      // [NSF][n1]
  C* stage = reinterpret_cast<C*>(smraw + lay.stage);    // [3*NR][P] raw rows of the next plane
  uint16_t* sids = reinterpret_cast<uint16_t*>(smraw + lay.ids);  // [2][TY+1][n1i]
  float* ssrc = reinterpret_cast<float*>(smraw + lay.src);        // [2][3*TY][n1s]
  T* edge = reinterpret_cast<T*>(smraw + lay.edge);      // [nwarps][TY+1][12]
  double* red = reinterpret_cast<double*>(smraw + lay.red);

  const int x = tid;
  const bool xact = x < n1;
  const int xm = (x == 0) ? n1 - 1 : x - 1;
  const int xr = xact ? x : 0, xmr = xact ? xm : 0;

  MarchPtrs<T> mp;
  mp.in = in;
  mp.ureal = a.ureal;
  mp.ids = ids;
  mp.src = a.src;
  mp.stage = stage;
  mp.rring = rring;
  mp.sids = sids;
  mp.ssrc = ssrc;
  mp.n1 = n1;
  mp.n2 = n2;
  mp.n3 = n3;
  mp.P = P;
  mp.y0 = y0;
  mp.n1i = lay.n1i;
  mp.n1s = lay.n1s;

  if (MODE == MODE_EMIT) {
    double* __restrict__ u64 = a.u64;
    march_prefetch<T, TY, REAL>(mp, tid, nthr, z0, 0, 0, -1, false);
    for (int p = z0; p < z0 + zc; ++p) {
      cp_async_wait_all();
      __syncthreads();
      march_pack<T, TY>(mp, ring, x, xact, 0);
      if (p + 1 < z0 + zc) march_prefetch<T, TY, REAL>(mp, tid, nthr, p + 1, 0, 0, -1, false);
      HS_FFT_ROWS(true, ring, rpitch(n1), NSI, plan, tw1, tid, nthr);
      __syncthreads();
      if (xact) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < TY; ++r)
            u64[c * rcomp + (size_t)p * rplane + (size_t)(y0 + r) * n1 + x] += (double)march_u<T, TY, REAL>(ring, rring, n1, 0, c, r + 1, x);
      }
      __syncthreads();
    }
    cp_async_wait_all();
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
  for (int i = 0; i < 6; ++i) E[i] = macro_E(a, i);

  const bool recv_shfl = (lane < 31) && (x + 1 < n1);
  const bool recv_edge = xact && !recv_shfl;
  const int src_warp = ((x + 1) % n1) >> 5;

  // prologue: plane z0-1, then the prefetch of plane z0
  if (REAL) {
    march_prefetch<T, TY, REAL>(mp, tid, nthr, z0 - 1, 0, 0, -1, false);
    march_prefetch<T, TY, REAL>(mp, tid, nthr, z0, 1, 0, -1, true);
  } else {
    march_prefetch<T, TY, REAL>(mp, tid, nthr, z0 - 1, 0, 0, -1, false);
    cp_async_wait_all();
    __syncthreads();
    march_pack<T, TY>(mp, ring, x, xact, 0);
    march_prefetch<T, TY, REAL>(mp, tid, nthr, z0, 0, 0, -1, true);
    HS_FFT_ROWS(true, ring, rpitch(n1), NSI, plan, tw1, tid, nthr);
    __syncthreads();
  }
  constexpr bool FORCE_LIKE = (MODE == MODE_FORCE || MODE == MODE_FORCE_FIELDS);
  const int pend = FORCE_LIKE ? z0 + zc : z0 + zc - 1;
  for (int p = z0; p <= pend; ++p) {
    const int ib = (p - z0) & 1;  // ids buffer of voxel plane p, source buffer of output plane p-1
    int sc, sp;
    cp_async_wait_all();
    __syncthreads();
    if (REAL) {
      sc = (p - z0 + 1) % 3;
      sp = (p - z0) % 3;
      if (p < pend) march_prefetch<T, TY, REAL>(mp, tid, nthr, p + 1, (p - z0 + 2) % 3, ib ^ 1, FORCE_LIKE ? p : -1, true);
    } else {
      sc = (p - z0 + 1) & 1;
      sp = sc ^ 1;
      march_pack<T, TY>(mp, ring, x, xact, sc);
      if (p < pend) march_prefetch<T, TY, REAL>(mp, tid, nthr, p + 1, 0, ib ^ 1, FORCE_LIKE ? p : -1, true);
      HS_FFT_ROWS(true, ring + sc * NSI * rpitch(n1), rpitch(n1), NSI, plan, tw1, tid, nthr);
      __syncthreads();
    }
    const int pz = p % n3;
    const bool own_plane = p < z0 + zc;
    const uint16_t* idrow = sids + (size_t)ib * (TY + 1) * lay.n1i;

    // ---- per-voxel work: rows jj = 1..TY+1 (voxel y = y0 + jj - 1) ----
    T uc[2][3][2];  // cached corner values of row jj: [ox][comp][oz]
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uc[0][c][0] = march_u<T, TY, REAL>(ring, rring, n1, sc, c, 0, xr);
      uc[0][c][1] = march_u<T, TY, REAL>(ring, rring, n1, sp, c, 0, xr);
      uc[1][c][0] = march_u<T, TY, REAL>(ring, rring, n1, sc, c, 0, xmr);
      uc[1][c][1] = march_u<T, TY, REAL>(ring, rring, n1, sp, c, 0, xmr);
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
        const T v00 = march_u<T, TY, REAL>(ring, rring, n1, sc, c, jj, xr);
        const T v01 = march_u<T, TY, REAL>(ring, rring, n1, sp, c, jj, xr);
        const T v10 = march_u<T, TY, REAL>(ring, rring, n1, sc, c, jj, xmr);
        const T v11 = march_u<T, TY, REAL>(ring, rring, n1, sp, c, jj, xmr);
        u[0][0][0][c] = v00; u[0][0][1][c] = v01; u[1][0][0][c] = v10; u[1][0][1][c] = v11;
        uc[0][c][0] = v00; uc[0][c][1] = v01; uc[1][c][0] = v10; uc[1][c][1] = v11;
      }
      const int yv = (y0 + jj - 1) % n2;
      const int ph = idrow[(size_t)(jj - 1) * lay.n1i + xr];
      if (MODE == MODE_FIELDS) {
        T e1[6], e2[6], s1[6], s2[6];
        tetra_strains(u, E, e1, e2);
        mat.stress(ph, e1, s1);
        mat.stress(ph, e2, s2);
        if (a.sig0 != nullptr) {
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            const T s0 = a.sig0[6 * ph + i];
            s1[i] -= s0;
            s2[i] -= s0;
          }
        }
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
      // F is accumulated as 4 F (the 1/4 of the adjoint is applied when a row is
      // complete); left-going vectors are sent with the sign their receiver applies.
#pragma unroll
      for (int tt = 0; tt < 2; ++tt) {
        T ev[6], sv[6];
        tetra_strain_fast(u, E, tt, ev);
        mat.stress(ph, ev, sv);
        if (a.sig0 != nullptr) {
#pragma unroll
          for (int i = 0; i < 6; ++i) sv[i] -= a.sig0[6 * ph + i];
        }
        if (!xact) {
#pragma unroll
          for (int i = 0; i < 6; ++i) sv[i] = 0;
        }
        if (acc_sig) {
#pragma unroll
          for (int i = 0; i < 6; ++i) sacc[i] += sv[i];
        }
        if constexpr (MODE == MODE_FORCE_FIELDS) {
          // eps = 1/2 (eps^T1 + eps^T2) (tensor components), sigma = 1/2 (sigma^T1 + sigma^T2):
          // T1's halves are stored, T2's added to them
          if (acc_sig) {
            const size_t o = (size_t)pz * rplane + (size_t)((y0 + jj - 1) % n2) * n1 + x;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
              const T eh = T(0.5) * ev[i] * (i < 3 ? T(1) : T(0.5));
              const T sh = T(0.5) * sv[i];
              if (a.out_f32) {
                float* ep = reinterpret_cast<float*>(a.eps_out) + i * rcomp + o;
                float* sp = reinterpret_cast<float*>(a.sig_out) + i * rcomp + o;
                if (tt == 0) { *ep = (float)eh; *sp = (float)sh; }
                else { *ep = (float)((T)*ep + eh); *sp = (float)((T)*sp + sh); }
              } else {
                double* ep = reinterpret_cast<double*>(a.eps_out) + i * rcomp + o;
                double* sp = reinterpret_cast<double*>(a.sig_out) + i * rcomp + o;
                if (tt == 0) { *ep = (double)eh; *sp = (double)sh; }
                else { *ep += (double)eh; *sp += (double)sh; }
              }
            }
          }
        }
        T l0[3], l1[3];
        // per force component k: (sigma_1k, sigma_2k, sigma_3k)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int i1 = (k == 0) ? 0 : (k == 1 ? 5 : 4);
          const int i2 = (k == 0) ? 5 : (k == 1 ? 1 : 3);
          const int i3 = (k == 0) ? 4 : (k == 1 ? 3 : 2);
          const T Ps = sv[i1] + sv[i2], Ms = sv[i1] - sv[i2], Zs = sv[i3];
          if (tt == 0) {
            if (jj - 1 < TY) Fn[jj - 1][k] += Ps + Zs;              // T1 a1 (0,0,0)
            if (jj - 2 >= 0) Fp[jj - 2][k] += Ms - Zs;              // T1 a2 (0,-1,-1)
            l0[k] = Zs - Ps;                                        // T1 a3 (-1,-1,0): +
            l1[k] = Ms + Zs;                                        // T1 a4 (-1,0,-1): -
          } else {
            if (jj - 2 >= 0) Fn[jj - 2][k] += Ms + Zs;              // T2 a3 (0,-1,0)
            if (jj - 1 < TY) Fp[jj - 1][k] += Ps - Zs;              // T2 a4 (0,0,-1)
            l0[k] = Ps + Zs;                                        // T2 a1 (-1,-1,-1): -
            l1[k] = Zs - Ms;                                        // T2 a2 (-1,0,0): +
          }
        }
        T g0[3], g1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          g0[k] = __shfl_down_sync(0xffffffffu, l0[k], 1);
          g1[k] = __shfl_down_sync(0xffffffffu, l1[k], 1);
        }
        if (lane == 0) {
          T* ed = edge + (warp * (TY + 1) + (jj - 1)) * 12 + tt * 6;
#pragma unroll
          for (int k = 0; k < 3; ++k) { ed[k] = l0[k]; ed[3 + k] = l1[k]; }
        }
        if (recv_shfl) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if (tt == 0) {
              if (jj - 2 >= 0) Fn[jj - 2][k] += g0[k];
              if (jj - 1 < TY) Fp[jj - 1][k] -= g1[k];
            } else {
              if (jj - 2 >= 0) Fp[jj - 2][k] -= g0[k];
              if (jj - 1 < TY) Fn[jj - 1][k] += g1[k];
            }
          }
        }
      }
    }
    if (MODE == MODE_FIELDS) continue;
    __syncthreads();
    if (recv_edge) {
#pragma unroll
      for (int jj = 1; jj <= TY + 1; ++jj)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T* e = edge + (src_warp * (TY + 1) + (jj - 1)) * 12;
          if (jj - 2 >= 0) Fn[jj - 2][k] += e[0 * 3 + k];   // T1 a3
          if (jj - 1 < TY) Fp[jj - 1][k] -= e[1 * 3 + k];   // T1 a4
          if (jj - 2 >= 0) Fp[jj - 2][k] -= e[2 * 3 + k];   // T2 a1
          if (jj - 1 < TY) Fn[jj - 1][k] += e[3 * 3 + k];   // T2 a2
        }
    }
    if (p > z0) {
      // corner plane p-1 is complete: undo the factor 4 of the accumulation
      const int zp = (p - 1) % n3;
#pragma unroll
      for (int r = 0; r < TY; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) Fp[r][k] *= T(0.25);
      if (has_src && xact) {
        const float* sr = ssrc + (size_t)ib * 3 * TY * lay.n1s;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < TY; ++r) Fp[r][c] += (T)sr[(size_t)(c * TY + r) * lay.n1s + x];
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
            for (int r = 0; r < TY; ++r) {
              const size_t o = c * rcomp + (size_t)zp * rplane + (size_t)(y0 + r) * n1 + x;
              if (a.fout_f32) reinterpret_cast<float*>(a.fout)[o] = (float)Fp[r][c];
              else reinterpret_cast<T*>(a.fout)[o] = Fp[r][c];
            }
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
              fbuf[((c * TY + r) >> 1) * rpitch(n1) + rpad(x)] = z;
            }
        }
        __syncthreads();
        HS_FFT_ROWS(false, fbuf, rpitch(n1), NSF, plan, tw1, tid, nthr);
        __syncthreads();
        if (x < nh) {
          const int k = x;
#pragma unroll
          for (int q = 0; q < NSF; ++q) {
            const C Zk = fbuf[q * rpitch(n1) + rpad(k)];
            const C Zn = fbuf[q * rpitch(n1) + rpad(k == 0 ? 0 : n1 - k)];
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
    }
#pragma unroll
    for (int r = 0; r < TY; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) { Fp[r][k] = Fn[r][k]; Fn[r][k] = 0; }
  }
  cp_async_wait_all();
  if (!FORCE_LIKE) return;
  double acc[NRED];
#pragma unroll
  for (int i = 0; i < 6; ++i) acc[i] = (double)sacc[i];
  acc[6] = (double)facc;
  reduce_and_finalize(acc, a.partials, a.st, a.hist, red);
}

}  // namespace hs
