// FP32 real-space pass of the basic scheme: strain stencil, constitutive step
// and adjoint stencil on a real displacement field, marching along z.
//
// Same contract as k_march with REAL = true (see march.cuh for the tiling and
// the plane/row conventions), organised for instruction count:
//
// * Both tetrahedra in one packed stream.  T2 is the point reflection of T1
//   through the voxel centre: with the T1 corners a = (0,0,0), b = (0,-1,-1),
//   c = (-1,-1,0), d = (-1,0,-1) (offsets from the voxel's upper corner; Eq.
//   DA1) and their mirror images a' = (-1,-1,-1), b' = (-1,0,0), c' = (0,0,-1),
//   d' = (0,-1,0), the pairs (u(a), u(a')), ... run through the T1 formulas
//   in the two lanes of f32x2 instructions: lane y then holds -2 D^T2 u
//   (Eqs. DA2, DB1), so the strain takes 1/2 in lane x and -1/2 in lane y.
//   Stress and the adjoint combinations are lane-wise; lane y's adjoint
//   contributions go to the mirrored corners with the opposite sign.
// * The force for column x-1 is collected per corner row in a two-row window
//   and sent once per completed row (6 values) by warp shuffle; lane 0 passes
//   its values to the previous warp's lane 31 through shared memory.
// * The prefetch maps warps to rows and lanes to 16-byte chunks, so the
//   per-plane copy needs no division.
#pragma once
#include "march.cuh"

namespace hs {

__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as one packed FMA (b * -1 is exact, so the result is the rounded difference)
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p2dup(float v) { return make_float2(v, v); }

// Packed constitutive laws: s = C(ph) : e for both lanes (engineering Voigt strain).
struct MatIsoP {
  const float* tab;  // (lambda, mu) per phase, 8-byte aligned
  __device__ __forceinline__ void stress(int ph, const float2 (&e)[6], float2 (&s)[6]) const {
    const float2 lm = __ldg(reinterpret_cast<const float2*>(tab) + ph);
    const float2 lam = p2dup(lm.x), mu = p2dup(lm.y), m2 = p2dup(lm.y + lm.y);
    const float2 lt = p2mul(lam, p2add(p2add(e[0], e[1]), e[2]));
    s[0] = p2fma(m2, e[0], lt);
    s[1] = p2fma(m2, e[1], lt);
    s[2] = p2fma(m2, e[2], lt);
    s[3] = p2mul(mu, e[3]);
    s[4] = p2mul(mu, e[4]);
    s[5] = p2mul(mu, e[5]);
  }
};

struct MatAnisoP {
  const float* tab;  // 21 upper-triangle Voigt entries per phase, row-major
  __device__ __forceinline__ void stress(int ph, const float2 (&e)[6], float2 (&s)[6]) const {
    const float* c = tab + 21 * ph;
    float C[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) C[i] = __ldg(c + i);
#define HS_UT(i, j) ((i) * 6 - ((i) * ((i) - 1)) / 2 + ((j) - (i)))
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float2 acc = p2mul(p2dup(C[HS_UT(0, i)]), e[0]);  // entry (i, 0) = (0, i)
#pragma unroll
      for (int j = 1; j < 6; ++j) acc = p2fma(p2dup(C[i <= j ? HS_UT(i, j) : HS_UT(j, i)]), e[j], acc);
      s[i] = acc;
    }
#undef HS_UT
  }
};

// Asynchronous prefetch of one plane: u rows of corner plane pu into ring slot
// `slot`, ids rows of voxel plane pu into buffer ib (if want_ids), source rows
// of output plane ps into buffer ib (ps < 0: none).  Warp w copies rows w,
// w + nwarps, ...; its lanes copy the 16-byte chunks of a row.  Ends with a
// commit of the copy group.
template <int TY, int N1>
__device__ __forceinline__ void stencil_prefetch(const MarchArgs<float>& a, const MarchLayout& lay,
                                                 unsigned char* smraw, int y0, int pu, int slot, int ib, int ps,
                                                 bool want_ids) {
  constexpr int NR = TY + 2;
  const int n1 = N1 > 0 ? N1 : a.n1, n2 = a.n2, n3 = a.n3;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const size_t rplane = (size_t)n2 * n1, rcomp = (size_t)n3 * rplane;
  const int gz = pu < 0 ? pu + n3 : (pu >= n3 ? pu - n3 : pu);
  float* dst0 = reinterpret_cast<float*>(smraw + lay.ring) + (size_t)slot * 3 * NR * n1;
  const float* srcz = a.ureal + (size_t)gz * rplane;
  if ((n1 & 3) == 0) {
    const int nch = n1 >> 2;
    for (int r = warp; r < 3 * NR; r += nw) {
      const int c = r / NR, j = r - c * NR;
      int gy = y0 - 1 + j;
      gy += (gy < 0) ? n2 : 0;
      gy -= (gy >= n2) ? n2 : 0;
      const float* s = srcz + c * rcomp + (size_t)gy * n1;
      float* d = dst0 + r * n1;
      for (int q = lane; q < nch; q += 32) cp_async16(d + 4 * q, s + 4 * q);
    }
  } else if (tid < n1) {
    for (int r = 0; r < 3 * NR; ++r) {
      const int c = r / NR, j = r - c * NR;
      const int gy = (y0 - 1 + j + n2) % n2;
      dst0[r * n1 + tid] = srcz[c * rcomp + (size_t)gy * n1 + tid];
    }
  }
  if (want_ids) {
    uint16_t* d0 = reinterpret_cast<uint16_t*>(smraw + lay.ids) + (size_t)ib * (TY + 1) * lay.n1i;
    const uint16_t* s0 = a.ids + (size_t)gz * n2 * n1;
    if ((n1 & 7) == 0) {
      const int nch = n1 >> 3;
      for (int r = warp; r <= TY; r += nw) {
        const int gy = (y0 + r) - ((y0 + r >= n2) ? n2 : 0);
        for (int q = lane; q < nch; q += 32) cp_async16(d0 + r * lay.n1i + 8 * q, s0 + (size_t)gy * n1 + 8 * q);
      }
    } else if (tid < n1) {
      for (int r = 0; r <= TY; ++r) d0[r * lay.n1i + tid] = s0[(size_t)((y0 + r) % n2) * n1 + tid];
    }
  }
  if (a.src != nullptr && ps >= 0) {
    float* d0 = reinterpret_cast<float*>(smraw + lay.src) + (size_t)ib * 3 * TY * lay.n1s;
    const float* s0 = a.src + (size_t)(ps % n3) * rplane;
    if ((n1 & 3) == 0) {
      const int nch = n1 >> 2;
      for (int r = warp; r < 3 * TY; r += nw) {
        const int c = r / TY, rr = r - c * TY;
        const float* s = s0 + c * rcomp + (size_t)(y0 + rr) * n1;
        for (int q = lane; q < nch; q += 32) cp_async16(d0 + r * lay.n1s + 4 * q, s + 4 * q);
      }
    } else if (tid < n1) {
      for (int r = 0; r < 3 * TY; ++r) {
        const int c = r / TY, rr = r - c * TY;
        d0[r * lay.n1s + tid] = s0[c * rcomp + (size_t)(y0 + rr) * n1 + tid];
      }
    }
  }
  cp_async_commit();
}

// One bulk copy of rows y, y + 1, ... of a plane (the rows of y0 + r0 .. y0 + r1 - 1, each
// wrapped into [0, n2)) into consecutive shared rows: split where the wrap breaks contiguity.
// Issued by one thread; completes on bar.
__device__ __forceinline__ void bulk_rows(unsigned char* dst, const unsigned char* plane, int y_first, int nrows,
                                          int n2, unsigned rowbytes, uint64_t* bar) {
  int y = y_first, r = 0;
  y += (y < 0) ? n2 : 0;
  y -= (y >= n2) ? n2 : 0;
  while (r < nrows) {
    const int run = min(nrows - r, n2 - y);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst + (size_t)r * rowbytes)),
                 "l"(plane + (size_t)y * rowbytes), "r"((unsigned)run * rowbytes), "r"(smem_u32(bar))
                 : "memory");
    r += run;
    y = 0;
  }
}

// The plane copies of stencil_prefetch as bulk copies by the calling thread (compile-time N1,
// a multiple of 8): per component one run of rows (two or three where y wraps), the id rows
// and the source rows likewise, all completing on the ring slot's mbarrier.
template <int TY, int N1>
__device__ __forceinline__ void stencil_prefetch_bulk(const MarchArgs<float>& a, const MarchLayout& lay,
                                                      unsigned char* smraw, int y0, int pu, int slot, int ib, int ps,
                                                      bool want_ids, uint64_t* bar) {
  constexpr int NR = TY + 2;
  const int n2 = a.n2, n3 = a.n3;
  const size_t rplane = (size_t)n2 * N1, rcomp = (size_t)n3 * rplane;
  const int gz = pu < 0 ? pu + n3 : (pu >= n3 ? pu - n3 : pu);
  const bool src = a.src != nullptr && ps >= 0;
  mbar_arrive_expect_tx(bar, (unsigned)(3 * NR * N1 * 4 + (want_ids ? (TY + 1) * N1 * 2 : 0) +
                                        (src ? 3 * TY * N1 * 4 : 0)));
  unsigned char* ring = smraw + lay.ring + (size_t)slot * 3 * NR * N1 * 4;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    bulk_rows(ring + (size_t)c * NR * N1 * 4,
              reinterpret_cast<const unsigned char*>(a.ureal + c * rcomp + (size_t)gz * rplane), y0 - 1, NR, n2,
              N1 * 4, bar);
  if (want_ids)
    bulk_rows(smraw + lay.ids + (size_t)ib * (TY + 1) * N1 * 2,
              reinterpret_cast<const unsigned char*>(a.ids + (size_t)gz * rplane), y0, TY + 1, n2, N1 * 2, bar);
  if (src) {
    const size_t zs = (size_t)(ps % n3) * rplane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      bulk_rows(smraw + lay.src + ((size_t)ib * 3 * TY + (size_t)c * TY) * N1 * 4,
                reinterpret_cast<const unsigned char*>(a.src + c * rcomp + zs), y0, TY, n2, N1 * 4, bar);
  }
}

// N1 > 0: the x extent is a compile-time constant (hot sizes), so shared
// memory row offsets become immediates; N1 = 0: taken at run time.
// BATCH: a batched launch (grid.z items, every workspace pointer moved per item);
// a single solve's launch uses the arguments as they come.
template <int TY, class MATP, int MODE, int N1 = 0, bool BATCH = false>
__global__ void __launch_bounds__(512) k_stencil(const MarchArgs<float> a_, const MATP mat_) {
  constexpr int NR = TY + 2;
  const MarchArgs<float> a = BATCH ? march_item_args(a_) : a_;
  MATP mat = mat_;
  if (BATCH) mat.tab = a.mat;
  if (a.st->retired || (a.skip_if_done && a.st->done)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n1 = N1 > 0 ? N1 : a.n1, n2 = a.n2, n3 = a.n3;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int y0 = blockIdx.x * TY;
  const int z0 = blockIdx.y * a.zc;
  const int zc = min(a.zc, n3 - z0);
  const size_t rplane = (size_t)n2 * n1;
  const size_t rcomp = (size_t)n3 * rplane;
  const bool has_src = (a.src != nullptr);

  const MarchLayout lay = march_layout(n1, 0, nthr, TY, MODE, true, has_src, 4);
  const int n1i = N1 > 0 ? ((N1 + 7) & ~7) : lay.n1i;
  const int n1s = N1 > 0 ? ((N1 + 3) & ~3) : lay.n1s;
  float* rring = reinterpret_cast<float*>(smraw + lay.ring);            // [3][3*NR][n1]
  uint16_t* sids = reinterpret_cast<uint16_t*>(smraw + lay.ids);        // [2][TY+1][n1i]
  float* ssrc = reinterpret_cast<float*>(smraw + lay.src);              // [2][3*TY][n1s]
  float* edge = reinterpret_cast<float*>(smraw + lay.edge);             // [nwarps][TY][6]
  double* red = reinterpret_cast<double*>(smraw + lay.red);

  const int x = tid;
  const bool xact = x < n1;
  const int xm = (x == 0) ? n1 - 1 : x - 1;
  const int xr = xact ? x : 0, xmr = xact ? xm : 0;

  float Fp[TY][3], Fn[TY][3];
#pragma unroll
  for (int r = 0; r < TY; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) { Fp[r][k] = 0.f; Fn[r][k] = 0.f; }
  float2 sacc[6];  // lane x: sum sigma^T1, lane y: sum sigma^T2
#pragma unroll
  for (int i = 0; i < 6; ++i) sacc[i] = make_float2(0.f, 0.f);
  float facc = 0.f;
  // 1/2 and -1/2 undo the packing
  const float2 hh = make_float2(0.5f, -0.5f);
  float Em[6];  // engineering macro strain
#pragma unroll
  for (int i = 0; i < 6; ++i) Em[i] = (i < 3 ? 1.f : 2.f) * macro_E(a, i);

  const bool recv_shfl = (lane < 31) && (x + 1 < n1);
  const bool recv_edge = xact && !recv_shfl;
  const int src_warp = ((x + 1) % n1) >> 5;

  // compile-time x extents (a multiple of 8): planes arrive by bulk copies from thread 0, plane
  // q in ring slot (q - z0 + 1) % 3 completing on that slot's mbarrier (waits bounded; a
  // timeout is recorded in the status)
  constexpr bool BULK = N1 > 0 && N1 % 8 == 0;
  uint64_t* const pbar = reinterpret_cast<uint64_t*>(smraw + lay.bar);
  bool timed_out = false;
  if (BULK) {
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) mbar_init(pbar + q, 1);
      mbar_init_fence();
      stencil_prefetch_bulk<TY, (BULK ? N1 : 8)>(a, lay, smraw, y0, z0 - 1, 0, 0, -1, false, pbar);
      stencil_prefetch_bulk<TY, (BULK ? N1 : 8)>(a, lay, smraw, y0, z0, 1, 0, -1, true, pbar + 1);
    }
    __syncthreads();  // the barriers are initialised before anyone waits on them
  } else {
    stencil_prefetch<TY, N1>(a, lay, smraw, y0, z0 - 1, 0, 0, -1, false);
    stencil_prefetch<TY, N1>(a, lay, smraw, y0, z0, 1, 0, -1, true);
  }

  const int pend = (MODE == MODE_FORCE) ? z0 + zc : z0 + zc - 1;
  for (int p = z0; p <= pend; ++p) {
    const int ib = (p - z0) & 1;
    const int sc = (p - z0 + 1) % 3, sp = (p - z0) % 3;
    if (BULK) {
      if (p == z0) timed_out |= !mbar_wait(pbar, 0);
      timed_out |= !mbar_wait(pbar + sc, (unsigned)(((p - z0 + 1) / 3) & 1));
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    if (p < pend) {
      if (BULK) {
        if (tid == 0)
          stencil_prefetch_bulk<TY, (BULK ? N1 : 8)>(a, lay, smraw, y0, p + 1, (p - z0 + 2) % 3, ib ^ 1,
                                                     MODE == MODE_FORCE ? p : -1, true, pbar + (p - z0 + 2) % 3);
      } else {
        stencil_prefetch<TY, N1>(a, lay, smraw, y0, p + 1, (p - z0 + 2) % 3, ib ^ 1, MODE == MODE_FORCE ? p : -1,
                                 true);
      }
    }
    const int pz = p % n3;
    const bool own_plane = p < z0 + zc;
    const uint16_t* idrow = sids + (size_t)ib * (TY + 1) * n1i;
    const float* rc = rring + (size_t)sc * 3 * NR * n1;  // corner plane p
    const float* rp = rring + (size_t)sp * 3 * NR * n1;  // corner plane p-1

    // corner values of ring row j: [own/left][plane p / p-1][comp]
    float un[2][2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      un[0][0][c] = rc[(c * NR) * n1 + xr];
      un[0][1][c] = rp[(c * NR) * n1 + xr];
      un[1][0][c] = rc[(c * NR) * n1 + xmr];
      un[1][1][c] = rp[(c * NR) * n1 + xmr];
    }
    // left-going force of corner rows jj-2 (W0) and jj-1 (W1): [plane p / p-1][comp]
    float W0[2][3], W1[2][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { W0[0][k] = W0[1][k] = W1[0][k] = W1[1][k] = 0.f; }

#pragma unroll
    for (int jj = 1; jj <= TY + 1; ++jj) {
      if (MODE == MODE_FIELDS && jj == TY + 1) break;
      // uo: previous ring row (oy = -1), un: this ring row (oy = 0)
      float uo[2][2][3];
#pragma unroll
      for (int ox = 0; ox < 2; ++ox)
#pragma unroll
        for (int oz = 0; oz < 2; ++oz)
#pragma unroll
          for (int c = 0; c < 3; ++c) uo[ox][oz][c] = un[ox][oz][c];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        un[0][0][c] = rc[(c * NR + jj) * n1 + xr];
        un[0][1][c] = rp[(c * NR + jj) * n1 + xr];
        un[1][0][c] = rc[(c * NR + jj) * n1 + xmr];
        un[1][1][c] = rp[(c * NR + jj) * n1 + xmr];
      }
      const int ph = idrow[(jj - 1) * n1i + xr];
      // T1 corner / mirror pairs: A = (000, 111), B = (011, 100), C = (110, 001), D = (101, 010)
      // with offset index [ox][oy][oz], 1 = coordinate - 1
      float2 g[3][3];  // g[i][j]: lane x = 2 D^T1_i u_j, lane y = -2 D^T2_i u_j
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float2 A = make_float2(un[0][0][j], uo[1][1][j]);
        const float2 B = make_float2(uo[0][1][j], un[1][0][j]);
        const float2 C = make_float2(uo[1][0][j], un[0][1][j]);
        const float2 D = make_float2(un[1][1][j], uo[0][0][j]);
        const float2 pp = p2add(A, B), qq = p2add(C, D), mm = p2sub(A, B), nn = p2sub(C, D);
        g[0][j] = p2sub(pp, qq);
        g[1][j] = p2sub(mm, nn);
        g[2][j] = p2add(mm, nn);
      }
      float2 e[6], s[6];
      e[0] = p2fma(hh, g[0][0], p2dup(Em[0]));
      e[1] = p2fma(hh, g[1][1], p2dup(Em[1]));
      e[2] = p2fma(hh, g[2][2], p2dup(Em[2]));
      e[3] = p2fma(hh, p2add(g[1][2], g[2][1]), p2dup(Em[3]));
      e[4] = p2fma(hh, p2add(g[0][2], g[2][0]), p2dup(Em[4]));
      e[5] = p2fma(hh, p2add(g[0][1], g[1][0]), p2dup(Em[5]));
      mat.stress(ph, e, s);
      if (a.sig0 != nullptr) {
#pragma unroll
        for (int i = 0; i < 6; ++i) s[i] = p2sub(s[i], p2dup(a.sig0[6 * ph + i]));
      }
      const int yv = y0 + jj - 1;
      if (MODE == MODE_FIELDS) {
        if (xact && own_plane) {
          const size_t o = (size_t)pz * rplane + (size_t)yv * n1 + x;
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            const float ev = 0.5f * (e[i].x + e[i].y) * (i < 3 ? 1.f : 0.5f);
            const float sv = 0.5f * (s[i].x + s[i].y);
            if (a.out_f32) {
              reinterpret_cast<float*>(a.eps_out)[i * rcomp + o] = ev;
              reinterpret_cast<float*>(a.sig_out)[i * rcomp + o] = sv;
            } else {
              reinterpret_cast<double*>(a.eps_out)[i * rcomp + o] = (double)ev;
              reinterpret_cast<double*>(a.sig_out)[i * rcomp + o] = (double)sv;
            }
          }
        }
        continue;
      }
      if (!xact) {
#pragma unroll
        for (int i = 0; i < 6; ++i) s[i] = make_float2(0.f, 0.f);
      }
      if (xact && own_plane && jj <= TY) {
#pragma unroll
        for (int i = 0; i < 6; ++i) sacc[i] = p2add(sacc[i], s[i]);
      }
      // adjoint: 4 F contributions per force component k from (sigma_1k, sigma_2k, sigma_3k)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int i1 = (k == 0) ? 0 : (k == 1 ? 5 : 4);
        const int i2 = (k == 0) ? 5 : (k == 1 ? 1 : 3);
        const int i3 = (k == 0) ? 4 : (k == 1 ? 3 : 2);
        const float2 Ps = p2add(s[i1], s[i2]), Ms = p2sub(s[i1], s[i2]);
        const float2 Pa = p2add(Ps, s[i3]);  // a: own (0,0,0) | a': left (-1,-1,-1), minus
        const float2 Pb = p2sub(Ms, s[i3]);  // b: own (0,-1,-1) | b': left (-1,0,0), minus
        const float2 Pc = p2sub(s[i3], Ps);  // c: left (-1,-1,0) | c': own (0,0,-1), minus
        const float2 Pd = p2add(Ms, s[i3]);  // d: left (-1,0,-1), minus | d': own (0,-1,0)
        if (jj - 1 < TY) {
          Fn[jj - 1][k] += Pa.x;
          Fp[jj - 1][k] -= Pc.y;
          W1[0][k] = -Pb.y;
          W1[1][k] = -Pd.x;
        }
        if (jj - 2 >= 0) {
          Fp[jj - 2][k] += Pb.x;
          Fn[jj - 2][k] += Pd.y;
          W0[0][k] += Pc.x;
          W0[1][k] -= Pa.y;
        }
      }
      // corner row jj-2 has all of this thread's left-going contributions: send them
      if (jj - 2 >= 0) {
        float g0[2][3];
#pragma unroll
        for (int z = 0; z < 2; ++z)
#pragma unroll
          for (int k = 0; k < 3; ++k) g0[z][k] = __shfl_down_sync(0xffffffffu, W0[z][k], 1);
        if (lane == 0) {
          float* ed = edge + (warp * TY + (jj - 2)) * 6;
          reinterpret_cast<float2*>(ed)[0] = make_float2(W0[0][0], W0[0][1]);
          reinterpret_cast<float2*>(ed)[1] = make_float2(W0[0][2], W0[1][0]);
          reinterpret_cast<float2*>(ed)[2] = make_float2(W0[1][1], W0[1][2]);
        }
        if (recv_shfl) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            Fn[jj - 2][k] += g0[0][k];
            Fp[jj - 2][k] += g0[1][k];
          }
        }
      }
#pragma unroll
      for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int k = 0; k < 3; ++k) { W0[z][k] = W1[z][k]; W1[z][k] = 0.f; }
    }
    if (MODE == MODE_FIELDS) continue;
    __syncthreads();
    if (recv_edge) {
#pragma unroll
      for (int r = 0; r < TY; ++r) {
        const float* e = edge + (src_warp * TY + r) * 6;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Fn[r][k] += e[k];
          Fp[r][k] += e[3 + k];
        }
      }
    }
    if (p > z0) {
      // corner plane p-1 is complete: undo the factor 4 of the accumulation
      const int zp = (p - 1) % n3;
      const float* sr = ssrc + (size_t)ib * 3 * TY * n1s;
#pragma unroll
      for (int r = 0; r < TY; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float f = 0.25f * Fp[r][c];
          if (has_src && xact) f += sr[(c * TY + r) * n1s + x];
          Fp[r][c] = f;
        }
      if (xact) {
        float* fo = reinterpret_cast<float*>(a.fout);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < TY; ++r) {
            facc = fmaf(Fp[r][c], Fp[r][c], facc);
            if (fo != nullptr) fo[c * rcomp + (size_t)zp * rplane + (size_t)(y0 + r) * n1 + x] = Fp[r][c];
          }
      }
    }
#pragma unroll
    for (int r = 0; r < TY; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) { Fp[r][k] = Fn[r][k]; Fn[r][k] = 0.f; }
  }
  cp_async_wait_all();
  if (BULK && timed_out) a.st->done = DONE_TIMEOUT;
  if (MODE != MODE_FORCE) return;
  double acc[NRED];
#pragma unroll
  for (int i = 0; i < 6; ++i) acc[i] = (double)sacc[i].x + (double)sacc[i].y;
  acc[6] = (double)facc;
  reduce_and_finalize(acc, a.partials, a.st, a.hist, red);
}

}  // namespace hs
