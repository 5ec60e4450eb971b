// FP32 real-space pass of the basic scheme on column pairs: strain stencil,
// constitutive step and adjoint stencil (Eqs. deps, DA1-DA2, der_E_dep_Q;
// Algorithm 1 step 3), every voxel computed once.
//
// Mapping.  A block owns R = RG * TY voxel rows y0 .. y0 + R - 1 of a chunk of
// z planes and all N1 columns, and marches along z.  Thread t of row group g
// (RG groups of NT threads) owns the column pair (2t, 2t + 1) and the voxel rows
// y0 + g TY .. y0 + g TY + TY - 1: every quantity is a float2 over the two
// columns, so one f32x2 instruction serves two voxels and the corner values of
// a pair arrive in one 8-byte shared-memory load.
//
// Corners.  Voxel (x, y, z) has the corners (x - ox, y - oy, z - oz), o in
// {0,1}^3 (corner (l+1/2, m+1/2, n+1/2) carries index (l, m, n)).  The first
// tetrahedron uses a = (0,0,0), b = (0,1,1), c = (1,1,0), d = (1,0,1) with
// 2 D_1 u = a + b - c - d, 2 D_2 u = (a - b) - (c - d), 2 D_3 u = (a - b) + (c - d)
// (Eq. DA1 term by term); the second the point reflections a' = (1,1,1),
// b' = (1,0,0), c' = (0,0,1), d' = (0,1,0) through the same formulas, which give
// -2 D^T2 u (Eqs. DB1, DA2).  Offset ox = 0 is the thread's own column pair,
// ox = 1 the pair shifted one column left (its first value read separately).
//
// Adjoint.  The nodal force F_k = dE/du_k gathers 1/4 sum_i c_i sigma_ik over
// the tetrahedra that contain the corner (c_i the stencil coefficient of the
// corner).  Contributions to the thread's own columns are added to float2
// accumulators of corner rows r = 0 .. TY (r = 0: the row below the group's
// rows) for the planes p - 1 (Fp) and p (Fn); contributions to column 2t - 1
// go to the left neighbour: summed per corner row and sent once the row is
// complete, by warp shuffle, or through shared memory across warps.
//
// Rows shared between groups and blocks.  Corner row y0 + g TY - 1 takes voxel
// rows of groups g - 1 and g: group g's part crosses to group g - 1 through
// shared memory when the plane completes, and group 0's part (the row below the
// block) is written to a side buffer that the forward x transform adds before
// it transforms that row.  So no voxel is computed twice across y.  In z the
// block computes one voxel plane past its chunk (the next chunk's first) to
// complete its last corner plane.
//
// Sums.  sum sigma^T1 + sigma^T2 over the block's own voxels is kept per plane
// in FP32 and carried across planes in compensated (Kahan) FP32 pairs, then
// reduced in FP64 into per-block partials.  |F|^2 is summed where F is complete:
// in the forward x transform, which also takes the stopping test (Eqs. L2-norm,
// tolerance) from both partial sums.
#pragma once
#include "stencil.cuh"

namespace hs {

// Planes in flight: the copy of plane p + XP_AHEAD starts when plane p is
// processed, so a block's short per-plane work does not wait for memory.
constexpr int XP_AHEAD = 3;
constexpr int XP_SLOTS = XP_AHEAD + 2;  // corner planes p - 1, p and the ones in flight
constexpr int XP_BUFS = XP_AHEAD + 1;   // ids and source planes

// Shared memory of k_xpair (host and device use the same function).
struct XpLayout {
  size_t ring, ids, src, edge, xchg, red, total;
};

__host__ __device__ inline XpLayout xp_layout(int n1, int nt, int rg, int ty, bool has_src) {
  XpLayout L;
  const int R = rg * ty;
  const int nw = (nt + 31) / 32;  // warps per row group
  size_t off = 0;
  L.ring = off;  // [XP_SLOTS][3 comps][R + 1 rows][n1] corner values
  off += hs_align16((size_t)4 * XP_SLOTS * 3 * (R + 1) * n1);
  L.ids = off;  // [XP_BUFS][R][n1] phase ids
  off += hs_align16((size_t)2 * XP_BUFS * R * ((n1 + 7) & ~7));
  L.src = off;  // [XP_BUFS][3][R][n1] correction source
  off += hs_align16(has_src ? (size_t)4 * XP_BUFS * 3 * R * n1 : 0);
  L.edge = off;  // [rg][nw][ty + 1][6] left-going sums of each warp's lane 0
  off += hs_align16((size_t)4 * rg * nw * (ty + 1) * 6);
  L.xchg = off;  // [rg][3][n1] a group's part of the corner row below it
  off += hs_align16((size_t)4 * rg * 3 * n1);
  L.red = off;
  off += 32 * NRED * 8;
  L.total = off;
  return L;
}

struct XpArgs {
  const float* ureal;    // displacement [3][n3][n2][n1]
  const uint16_t* ids;   // [n3][n2][n1]
  const float* mat;      // phase table (MatIsoP / MatAnisoP layout)
  float* fout;           // force [3][n3][n2][n1]: own rows complete, a block's top row partial
  float* side;           // [3][n3][n2 / R][n1]: row y0 - 1 of each block, this block's part
  const float* src;      // correction source added to F (refined correction solves), or null
  double* partials;      // per block: sum sigma (6), in blocks of NRED doubles
  DevStatus* st;
  const double* Edev;    // macroscopic strain read here (null: E)
  const float* sig0;     // eigenstress per phase, or null
  float E[6];
  int n1, n2, n3, zc;
  int skip_if_done;
  size_t zstride;        // batched launches: bytes between the workspaces of consecutive items
};

__device__ __forceinline__ XpArgs xp_item_args(const XpArgs& a) {
  if (a.zstride == 0) return a;
  XpArgs b = a;
  const size_t o = (size_t)blockIdx.z * a.zstride;
  b.ureal = zshift(a.ureal, o);
  b.ids = zshift(a.ids, o);
  b.mat = zshift(a.mat, o);
  b.fout = zshift(a.fout, o);
  b.side = zshift(a.side, o);
  b.src = zshift(a.src, o);
  b.partials = zshift(a.partials, o);
  b.st = zshift(a.st, o);
  b.Edev = zshift(a.Edev, o);
  b.sig0 = zshift(a.sig0, o);
  return b;
}

// constitutive laws on a column pair: voxel 2t in lane x, 2t + 1 in lane y
struct XpIso {
  const float* tab;  // (lambda, mu) per phase
  __device__ __forceinline__ void load(int ph0, int ph1, float2 (&c)[2]) const {
    const float2 a = __ldg(reinterpret_cast<const float2*>(tab) + ph0);
    const float2 b = __ldg(reinterpret_cast<const float2*>(tab) + ph1);
    c[0] = make_float2(a.x, b.x);  // lambda
    c[1] = make_float2(a.y, b.y);  // mu
  }
  __device__ __forceinline__ void stress(const float2 (&c)[2], const float2 (&e)[6], float2 (&s)[6]) const {
    const float2 lt = p2mul(c[0], p2add(p2add(e[0], e[1]), e[2]));
    const float2 m2 = p2add(c[1], c[1]);
    s[0] = p2fma(m2, e[0], lt);
    s[1] = p2fma(m2, e[1], lt);
    s[2] = p2fma(m2, e[2], lt);
    s[3] = p2mul(c[1], e[3]);
    s[4] = p2mul(c[1], e[4]);
    s[5] = p2mul(c[1], e[5]);
  }
  static constexpr int NC = 2;
};

struct XpAniso {
  const float* tab;  // 21 upper-triangle Voigt entries per phase
  __device__ __forceinline__ void load(int ph0, int ph1, float2 (&c)[21]) const {
    const float* a = tab + 21 * ph0;
    const float* b = tab + 21 * ph1;
#pragma unroll
    for (int i = 0; i < 21; ++i) c[i] = make_float2(__ldg(a + i), __ldg(b + i));
  }
  __device__ __forceinline__ void stress(const float2 (&c)[21], const float2 (&e)[6], float2 (&s)[6]) const {
#define HS_UT(i, j) ((i) * 6 - ((i) * ((i) - 1)) / 2 + ((j) - (i)))
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float2 acc = p2mul(c[HS_UT(0, i)], e[0]);
#pragma unroll
      for (int j = 1; j < 6; ++j) acc = p2fma(c[i <= j ? HS_UT(i, j) : HS_UT(j, i)], e[j], acc);
      s[i] = acc;
    }
#undef HS_UT
  }
  static constexpr int NC = 21;
};

// Compensated accumulation (Kahan): s + c holds the running sum.
__device__ __forceinline__ void kahan2(float2& s, float2& c, float2 x) {
  const float2 y = p2sub(x, c);
  const float2 t = p2add(s, y);
  c = p2sub(p2sub(t, s), y);
  s = t;
}

// Strain of one tetrahedron from its four corner pairs (A, B, C, D in the
// order of a, b, c, d), engineering Voigt, for both columns:
// e = E + h * sym(2 D u) with h = 1/2 (first tetrahedron) or -1/2 (second).
__device__ __forceinline__ void xp_strain(const float2 (&A)[3], const float2 (&B)[3], const float2 (&C)[3],
                                          const float2 (&D)[3], const float2 (&Em)[6], float h, float2 (&e)[6]) {
  float2 g[3][3];  // g[i][j] = +-2 D_i u_j
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float2 pp = p2add(A[j], B[j]), qq = p2add(C[j], D[j]), mm = p2sub(A[j], B[j]), nn = p2sub(C[j], D[j]);
    g[0][j] = p2sub(pp, qq);
    g[1][j] = p2sub(mm, nn);
    g[2][j] = p2add(mm, nn);
  }
  const float2 hh = p2dup(h);
  e[0] = p2fma(hh, g[0][0], Em[0]);
  e[1] = p2fma(hh, g[1][1], Em[1]);
  e[2] = p2fma(hh, g[2][2], Em[2]);
  e[3] = p2fma(hh, p2add(g[1][2], g[2][1]), Em[3]);
  e[4] = p2fma(hh, p2add(g[0][2], g[2][0]), Em[4]);
  e[5] = p2fma(hh, p2add(g[0][1], g[1][0]), Em[5]);
}

// Asynchronous copy of one plane: u rows y0 - 1 .. y0 + R - 1 of corner plane
// pu into ring slot `slot`, ids rows of voxel plane pu into ids buffer ib (ib < 0:
// none), source rows of output plane ps into source buffer sb (ps < 0: none).
// Warps take rows, lanes the 16-byte chunks of a row.  Commits one copy group.
template <int TY>
__device__ __forceinline__ void xp_prefetch(const XpArgs& a, const XpLayout& lay, unsigned char* smraw, int R,
                                            int y0, int pu, int slot, int ib, int ps, int sb) {
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const size_t rplane = (size_t)n2 * n1, rcomp = (size_t)n3 * rplane;
  const int gz = pu < 0 ? pu + n3 : (pu >= n3 ? pu - n3 : pu);
  const int NRW = R + 1;
  float* dst0 = reinterpret_cast<float*>(smraw + lay.ring) + (size_t)slot * 3 * NRW * n1;
  const float* srcz = a.ureal + (size_t)gz * rplane;
  const int n1i = (n1 + 7) & ~7;
  if ((n1 & 3) == 0) {
    const int nch = n1 >> 2;
    for (int r = warp; r < 3 * NRW; r += nw) {
      const int c = r / NRW, j = r - c * NRW;
      int gy = y0 - 1 + j;
      gy += (gy < 0) ? n2 : 0;
      const float* s = srcz + c * rcomp + (size_t)gy * n1;
      float* d = dst0 + (size_t)r * n1;
      for (int q = lane; q < nch; q += 32) cp_async16(d + 4 * q, s + 4 * q);
    }
    if (ib >= 0) {
      uint16_t* di = reinterpret_cast<uint16_t*>(smraw + lay.ids) + (size_t)ib * R * n1i;
      const uint16_t* si = a.ids + (size_t)gz * rplane;
      if ((n1 & 7) == 0) {
        const int nci = n1 >> 3;
        for (int r = warp; r < R; r += nw)
          for (int q = lane; q < nci; q += 32) cp_async16(di + r * n1i + 8 * q, si + (size_t)(y0 + r) * n1 + 8 * q);
      } else {
        for (int r = warp; r < R; r += nw)
          for (int q = lane; q < n1; q += 32) di[r * n1i + q] = si[(size_t)(y0 + r) * n1 + q];
      }
    }
    if (a.src != nullptr && ps >= 0) {
      float* ds = reinterpret_cast<float*>(smraw + lay.src) + (size_t)sb * 3 * R * n1;
      const float* s0 = a.src + (size_t)ps * rplane;
      for (int r = warp; r < 3 * R; r += nw) {
        const int c = r / R, rr = r - c * R;
        const float* s = s0 + c * rcomp + (size_t)(y0 + rr) * n1;
        for (int q = lane; q < nch; q += 32) cp_async16(ds + (size_t)r * n1 + 4 * q, s + 4 * q);
      }
    }
  } else {
    // rows whose length is not a multiple of 4 floats: element copies
    for (int r = warp; r < 3 * NRW; r += nw) {
      const int c = r / NRW, j = r - c * NRW;
      const int gy = (y0 - 1 + j + n2) % n2;
      for (int q = lane; q < n1; q += 32) dst0[(size_t)r * n1 + q] = srcz[c * rcomp + (size_t)gy * n1 + q];
    }
    if (ib >= 0) {
      uint16_t* di = reinterpret_cast<uint16_t*>(smraw + lay.ids) + (size_t)ib * R * n1i;
      const uint16_t* si = a.ids + (size_t)gz * rplane;
      for (int r = warp; r < R; r += nw)
        for (int q = lane; q < n1; q += 32) di[r * n1i + q] = si[(size_t)(y0 + r) * n1 + q];
    }
    if (a.src != nullptr && ps >= 0) {
      float* ds = reinterpret_cast<float*>(smraw + lay.src) + (size_t)sb * 3 * R * n1;
      const float* s0 = a.src + (size_t)ps * rplane;
      for (int r = warp; r < 3 * R; r += nw) {
        const int c = r / R, rr = r - c * R;
        for (int q = lane; q < n1; q += 32) ds[(size_t)r * n1 + q] = s0[c * rcomp + (size_t)(y0 + rr) * n1 + q];
      }
    }
  }
  cp_async_commit();
}

// One launch: grid (N2 / R, z chunks[, items]); block RG * NT threads, NT =
// round-up(N1 / 2, 32).  MODE_FORCE only (fields come from k_stencil).
template <int TY, class MAT>
__global__ void __launch_bounds__(512) k_xpair(const XpArgs a_, const MAT mat_) {
  const XpArgs a = xp_item_args(a_);
  MAT mat = mat_;
  mat.tab = a.mat;
  if (a.st->retired || (a.skip_if_done && a.st->done)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const int NT = ((n1 / 2 + 31) / 32) * 32;
  const int RG = blockDim.x / NT;
  const int R = RG * TY, NRW = R + 1;
  const int tid = threadIdx.x, lane = tid & 31;
  const int g = tid / NT, t = tid - g * NT;
  const int nwg = NT / 32, wg = t >> 5;  // warps per group, warp within the group
  const int y0 = blockIdx.x * R;
  const int z0 = blockIdx.y * a.zc;
  const int zc = min(a.zc, n3 - z0);
  const size_t rplane = (size_t)n2 * n1, rcomp = (size_t)n3 * rplane;
  const bool has_src = (a.src != nullptr);
  const XpLayout lay = xp_layout(n1, NT, RG, TY, has_src);
  const float* ring = reinterpret_cast<const float*>(smraw + lay.ring);
  const uint16_t* sids = reinterpret_cast<const uint16_t*>(smraw + lay.ids);
  const float* ssrc = reinterpret_cast<const float*>(smraw + lay.src);
  float* edge = reinterpret_cast<float*>(smraw + lay.edge);
  float* xchg = reinterpret_cast<float*>(smraw + lay.xchg);
  double* red = reinterpret_cast<double*>(smraw + lay.red);
  const int n1i = (n1 + 7) & ~7;

  const int x0 = 2 * t;
  const bool xact = x0 < n1;
  const int xo = xact ? x0 : 0;                // own pair (x0, x0 + 1)
  const int xm = (xo == 0) ? n1 - 1 : xo - 1;  // the column left of the pair
  const int npair = n1 / 2;
  // left-going sums of this thread go to thread t - 1 (t = 0: to the last pair); a
  // thread receives from t + 1 by shuffle inside its warp, else through shared memory
  const bool recv_shfl = (lane < 31) && (t + 1 < npair);
  const bool recv_edge = xact && !recv_shfl;
  const int src_wg = ((t + 1) % npair) >> 5;

  float2 Em[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float v = (i < 3 ? 1.f : 2.f) * (a.Edev != nullptr ? (float)a.Edev[i] : a.E[i]);
    Em[i] = p2dup(v);
  }
  // accumulators (4 F) of corner rows r = 0 .. TY: ring row g TY + r
  float2 Fp[TY + 1][3], Fn[TY + 1][3];
#pragma unroll
  for (int r = 0; r <= TY; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) Fp[r][k] = Fn[r][k] = make_float2(0.f, 0.f);
  // sum of sigma^T1 + sigma^T2 over own voxels: FP32 within a plane (pls), carried across
  // planes in compensated FP32 (ssum + scmp)
  float2 ssum[6], scmp[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) ssum[i] = scmp[i] = make_float2(0.f, 0.f);

  // pipeline: corner plane q in ring slot (q - z0 + 1) % XP_SLOTS, ids of voxel plane q in
  // buffer (q - z0) % XP_BUFS, source of output plane q in buffer (q - z0) % XP_BUFS; one
  // copy group per plane (empty past the chunk), so that plane p is complete once at most
  // XP_AHEAD - 1 later groups are pending
  const int pend = z0 + zc;
  xp_prefetch<TY>(a, lay, smraw, R, y0, z0 - 1, 0, -1, -1, 0);
  for (int q = z0; q < z0 + XP_AHEAD - 1; ++q) {
    if (q <= pend) xp_prefetch<TY>(a, lay, smraw, R, y0, q, (q - z0 + 1) % XP_SLOTS, (q - z0) % XP_BUFS,
                                   q - 1 >= z0 ? q - 1 : -1, (q - 1 - z0 + XP_BUFS) % XP_BUFS);
    else cp_async_commit();
  }
  for (int p = z0; p <= pend; ++p) {
    {
      // plane p + XP_AHEAD - 1 goes into the slot of plane p - 3 (its ids and source buffers held
      // planes p - 2 and p - 3): all were last read during step p - 2, before the barriers of
      // step p - 1; then wait for plane p
      const int q = p + XP_AHEAD - 1;
      if (q <= pend) xp_prefetch<TY>(a, lay, smraw, R, y0, q, (q - z0 + 1) % XP_SLOTS, (q - z0) % XP_BUFS, q - 1,
                                     (q - 1 - z0) % XP_BUFS);
      else cp_async_commit();
      asm volatile("cp.async.wait_group %0;\n" ::"n"(XP_AHEAD - 1) : "memory");
      __syncthreads();
    }
    const int sc = (p - z0 + 1) % XP_SLOTS, sp = (p - z0) % XP_SLOTS;
    const bool own_plane = p < z0 + zc;
    const float* rc = ring + (size_t)sc * 3 * NRW * n1;  // corner plane p
    const float* rp = ring + (size_t)sp * 3 * NRW * n1;  // corner plane p - 1
    const uint16_t* idp = sids + (size_t)((p - z0) % XP_BUFS) * R * n1i;

    float2 pls[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) pls[i] = make_float2(0.f, 0.f);
    // corner pairs of the previous ring row (oy = 1): own and left, planes p / p - 1
    float2 oP[3], oQ[3], lP[3], lQ[3];
    {
      const int rr = g * TY;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float* rowc = rc + (size_t)(c * NRW + rr) * n1;
        const float* rowp = rp + (size_t)(c * NRW + rr) * n1;
        oP[c] = *reinterpret_cast<const float2*>(rowc + xo);
        oQ[c] = *reinterpret_cast<const float2*>(rowp + xo);
        lP[c] = make_float2(rowc[xm], oP[c].x);
        lQ[c] = make_float2(rowp[xm], oQ[c].x);
      }
    }
    // left-going sums of corner rows jj - 1 (W0) and jj (W1), planes p ([0]) / p - 1 ([1])
    float W0[2][3], W1[2][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) W0[0][k] = W0[1][k] = W1[0][k] = W1[1][k] = 0.f;

#pragma unroll
    for (int jj = 1; jj <= TY; ++jj) {
      const int rr = g * TY + jj;  // ring row of corner row y (this voxel row)
      float2 nP[3], nQ[3], mP[3], mQ[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float* rowc = rc + (size_t)(c * NRW + rr) * n1;
        const float* rowp = rp + (size_t)(c * NRW + rr) * n1;
        nP[c] = *reinterpret_cast<const float2*>(rowc + xo);
        nQ[c] = *reinterpret_cast<const float2*>(rowp + xo);
        mP[c] = make_float2(rowc[xm], nP[c].x);
        mQ[c] = make_float2(rowp[xm], nQ[c].x);
      }
      const uint32_t ph2 = *reinterpret_cast<const uint32_t*>(idp + (size_t)(rr - 1) * n1i + xo);
      float2 cm[MAT::NC];
      mat.load((int)(ph2 & 0xffffu), (int)(ph2 >> 16), cm);
#pragma unroll
      for (int tt = 0; tt < 2; ++tt) {
        // tt = 0, first tetrahedron: a own (y, p), b own (y-1, p-1), c left (y-1, p), d left (y, p-1);
        // tt = 1, second: a' left (y-1, p-1), b' left (y, p), c' own (y, p-1), d' own (y-1, p)
        float2 s[6];
        {
          float2 e[6];
          if (tt == 0) xp_strain(nP, oQ, lP, mQ, Em, 0.5f, e);
          else xp_strain(lQ, mP, nQ, oP, Em, -0.5f, e);
          mat.stress(cm, e, s);
        }
        if (a.sig0 != nullptr) {
          const float* q0 = a.sig0 + 6 * (ph2 & 0xffffu);
          const float* q1 = a.sig0 + 6 * (ph2 >> 16);
#pragma unroll
          for (int i = 0; i < 6; ++i) s[i] = p2sub(s[i], make_float2(q0[i], q1[i]));
        }
        if (!xact) {
#pragma unroll
          for (int i = 0; i < 6; ++i) s[i] = make_float2(0.f, 0.f);
        }
        if (own_plane) {
#pragma unroll
          for (int i = 0; i < 6; ++i) pls[i] = p2add(pls[i], s[i]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int i1 = (k == 0) ? 0 : (k == 1 ? 5 : 4);
          const int i2 = (k == 0) ? 5 : (k == 1 ? 1 : 3);
          const int i3 = (k == 0) ? 4 : (k == 1 ? 3 : 2);
          const float2 P = p2add(s[i1], s[i2]), M = p2sub(s[i1], s[i2]);
          const float2 qa = p2add(P, s[i3]);  // corner a: first tetrahedron own (y, p) +,  second left (y-1, p-1) -
          const float2 qb = p2sub(M, s[i3]);  // corner b: first own (y-1, p-1) +,          second left (y, p) -
          const float2 qc = p2sub(s[i3], P);  // corner c: first left (y-1, p) +,           second own (y, p-1) -
          const float2 qd = p2add(M, s[i3]);  // corner d: first left (y, p-1) -,           second own (y-1, p) +
          // left pairs: lane y is the own column x0, lane x goes to column x0 - 1
          if (tt == 0) {
            Fn[jj][k] = p2add(Fn[jj][k], qa);
            Fp[jj - 1][k] = p2add(Fp[jj - 1][k], qb);
            Fn[jj - 1][k].x += qc.y;
            Fp[jj][k].x -= qd.y;
            W0[0][k] += qc.x;
            W1[1][k] -= qd.x;
          } else {
            Fp[jj][k] = p2sub(Fp[jj][k], qc);
            Fn[jj - 1][k] = p2add(Fn[jj - 1][k], qd);
            Fp[jj - 1][k].x -= qa.y;
            Fn[jj][k].x -= qb.y;
            W0[1][k] -= qa.x;
            W1[0][k] -= qb.x;
          }
        }
      }
      // corner row jj - 1 has all of this group's left-going sums: send them (and row TY at the end)
#pragma unroll
      for (int last = 0; last < 2; ++last) {
        if (last == 1 && jj != TY) break;
        const int r = jj - 1 + last;
        float (&W)[2][3] = last ? W1 : W0;
        float gs[2][3];
#pragma unroll
        for (int z = 0; z < 2; ++z)
#pragma unroll
          for (int k = 0; k < 3; ++k) gs[z][k] = __shfl_down_sync(0xffffffffu, W[z][k], 1);
        if (lane == 0) {
          float* ed = edge + ((size_t)(g * nwg + wg) * (TY + 1) + r) * 6;
#pragma unroll
          for (int z = 0; z < 2; ++z)
#pragma unroll
            for (int k = 0; k < 3; ++k) ed[3 * z + k] = W[z][k];
        }
        if (recv_shfl) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            Fn[r][k].y += gs[0][k];
            Fp[r][k].y += gs[1][k];
          }
        }
      }
#pragma unroll
      for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          W0[z][k] = W1[z][k];
          W1[z][k] = 0.f;
        }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        oP[c] = nP[c];
        oQ[c] = nQ[c];
        lP[c] = mP[c];
        lQ[c] = mQ[c];
      }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) kahan2(ssum[i], scmp[i], pls[i]);
    __syncthreads();
    if (recv_edge) {
#pragma unroll
      for (int r = 0; r <= TY; ++r) {
        const float* e = edge + ((size_t)(g * nwg + src_wg) * (TY + 1) + r) * 6;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Fn[r][k].y += e[k];
          Fp[r][k].y += e[3 + k];
        }
      }
    }
    if (p > z0) {
      // corner plane p - 1 is complete but for the rows shared with the group below
      const int zp = (p - 1) % n3;
      if (xact) {
        float2* xg = reinterpret_cast<float2*>(xchg + (size_t)g * 3 * n1);
#pragma unroll
        for (int k = 0; k < 3; ++k) xg[k * npair + t] = Fp[0][k];
      }
      __syncthreads();
      if (xact) {
        if (g + 1 < RG) {
          const float2* xu = reinterpret_cast<const float2*>(xchg + (size_t)(g + 1) * 3 * n1);
#pragma unroll
          for (int k = 0; k < 3; ++k) Fp[TY][k] = p2add(Fp[TY][k], xu[k * npair + t]);
        }
        const float2 q = p2dup(0.25f);
        if (g == 0) {
          // row y0 - 1: this block's part, completed by the forward x transform
          const size_t so = (size_t)zp * (n2 / R) * n1 + (size_t)blockIdx.x * n1 + xo;
#pragma unroll
          for (int k = 0; k < 3; ++k)
            *reinterpret_cast<float2*>(a.side + (size_t)k * n3 * (n2 / R) * n1 + so) = p2mul(q, Fp[0][k]);
        }
        const float* sr = ssrc + (size_t)((p - 1 - z0) % XP_BUFS) * 3 * R * n1;
#pragma unroll
        for (int r = 1; r <= TY; ++r) {
          const int yr = y0 + g * TY + r - 1;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            float2 f = p2mul(q, Fp[r][k]);
            if (has_src) f = p2add(f, *reinterpret_cast<const float2*>(sr + (size_t)(k * R + g * TY + r - 1) * n1 + xo));
            *reinterpret_cast<float2*>(a.fout + k * rcomp + (size_t)zp * rplane + (size_t)yr * n1 + xo) = f;
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r <= TY; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Fp[r][k] = Fn[r][k];
        Fn[r][k] = make_float2(0.f, 0.f);
      }
  }
  cp_async_wait_all();
  // block sums of sigma^T1 + sigma^T2 (FP64), as this block's partials
  double acc[6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
    acc[i] = ((double)ssum[i].x - (double)scmp[i].x) + ((double)ssum[i].y - (double)scmp[i].y);
  const int nw = blockDim.x >> 5, warp = tid >> 5;
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    const double s = warp_sum(acc[v]);
    if (lane == 0) red[warp * NRED + v] = s;
  }
  __syncthreads();
  if (tid < 6) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += red[w * NRED + tid];
    a.partials[(size_t)(blockIdx.y * gridDim.x + blockIdx.x) * NRED + tid] = s;
  }
}

}  // namespace hs
