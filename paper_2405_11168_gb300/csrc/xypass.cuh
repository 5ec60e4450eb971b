// Fused x and y transforms of one (component, z plane) in a thread-block
// cluster: the half-spectrum plane between the two transforms never leaves
// the chip.
//
// XY_FWD: real force rows -> forward x FFT (two real rows per complex
//   sequence, as ROW_R2C) -> forward y FFT of every x-frequency column ->
//   half spectrum [3][n3][n2][P] (the input of the z pass).
// XY_INV: the z pass's output -> inverse y FFT -> inverse x FFT (Hermitian
//   extension of two half-spectrum rows, as ROW_C2R) -> real rows
//   [3][n3][n2][n1] (the real-space pass's displacement).
//
// One cluster of CS blocks owns one (component, z) plane.  Block r holds
// rows y in [r*RY, (r+1)*RY), RY = n2/CS, during the x transform and
// x-frequency columns [r*CB, r*CB + nc_r) during the y transform, CB = n1/(2 CS)
// and nc_r = CB (+1 for the last block, which also takes the Nyquist column
// n1/2).  Between the two, every block reads its part of the other blocks'
// shared memory (distributed shared memory), once per element.  The
// arithmetic of every transform is the one of the split passes (same plans,
// twiddles and operation order), so both pipelines give the same values.
//
// Skip rules are those of the split passes: a retired item or a finished
// solve (skip_if_done) returns at entry; the flag is read by every block of
// the cluster from a status that no kernel of this launch writes, so either
// every block of a cluster returns there or none does, and every cluster
// barrier is reached by all of them.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"

namespace hs {

enum { XY_FWD = 0, XY_INV = 1 };

struct XYArgs {
  const float* real_in;  // XY_FWD: real rows [3][n3][n2][n1]
  float* real_out;       // XY_INV: real rows
  float2* spec;          // half spectrum [3][n3][n2][P]: written by XY_FWD, read by XY_INV
  const float2* tw1;     // w_N1^j
  const float2* tw2;     // w_N2^j
  int n3, P;
  const DevStatus* st;
  int skip_if_done;
};

// Compile-time shape of the fused pass for an n1 x n2 plane and clusters of CS blocks.
template <int L1, int L2, int CS> struct XYShape {
  static constexpr int RY = L2 / CS;           // rows per block in the x transform
  static constexpr int NSEQ = RY / 2;          // complex sequences (row pairs) per block
  static constexpr int NH = L1 / 2 + 1;        // x frequencies
  static constexpr int CB = L1 / (2 * CS);     // columns per block in the y transform (last block: CB + 1)
  static constexpr int W = CB + 1;             // column slots of the y tile
  static constexpr int XP = NH;                // pitch of the x-spectrum rows
  static constexpr int T1 = L1 / kE, T2 = L2 / kE;
  static constexpr int NT_X = NSEQ * T1, NT_Y = W * T2;
  static constexpr int NT = ((NT_X > NT_Y ? NT_X : NT_Y) + 31) / 32 * 32;
  // shared memory: x-spectrum rows [RY][XP], y tile [L2][W], x sequences [NSEQ][L1] (swizzled)
  static constexpr size_t XBYTES = (size_t)RY * XP * 8;
  static constexpr size_t YBYTES = (size_t)L2 * W * 8;
  static constexpr size_t ZBYTES = (size_t)NSEQ * L1 * 8;
  static constexpr size_t XOFF = 0;
  static constexpr size_t YOFF = (XBYTES + 15) / 16 * 16;
  // XY_FWD: the x sequences are dead before the y tile is filled, so they share its space
  static constexpr size_t ZOFF_FWD = YOFF;
  static constexpr size_t SMEM_FWD = YOFF + (YBYTES > ZBYTES ? YBYTES : ZBYTES);
  // XY_INV: other blocks read the y tile while the x sequences are built, so both are kept
  static constexpr size_t ZOFF_INV = YOFF + (YBYTES + 15) / 16 * 16;
  static constexpr size_t SMEM_INV = ZOFF_INV + ZBYTES;
  static_assert(L2 % CS == 0 && RY % 2 == 0, "rows must split into pairs per block");
  static_assert(L1 % (2 * CS) == 0, "x frequencies must split evenly");
  static_assert(NSEQ * T1 <= NT && W * T2 <= NT, "one pass per transform");
};

// release/acquire halves of the cluster barrier (every thread of every block arrives)
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

template <int L1, int L2, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(XYShape<L1, L2, CS>::NT, 2)
    k_xy_fwd(const XYArgs a) {
  using S = XYShape<L1, L2, CS>;
  constexpr int NT = S::NT, RY = S::RY, NSEQ = S::NSEQ, W = S::W, XP = S::XP, CB = S::CB, NH = S::NH;
  if (a.st->retired || (a.skip_if_done && a.st->done)) return;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* X = reinterpret_cast<float2*>(smraw + S::XOFF);
  float2* Y = reinterpret_cast<float2*>(smraw + S::YOFF);
  float2* Z = reinterpret_cast<float2*>(smraw + S::ZOFF_FWD);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = (int)cl.block_rank();
  const size_t unit = blockIdx.x / CS;  // comp * n3 + z
  const size_t P = (size_t)a.P;

  // 1. real rows 2s, 2s+1 (s = warp) -> complex sequence s, straight from global memory
  if (warp < NSEQ) {
    const float* ra = a.real_in + (unit * L2 + (size_t)r * RY + 2 * warp) * L1;
    const float* rb = ra + L1;
    float4 va[L1 / 128], vb[L1 / 128];
#pragma unroll
    for (int q = 0; q < L1 / 128; ++q) {
      va[q] = __ldg(reinterpret_cast<const float4*>(ra) + lane + 32 * q);
      vb[q] = __ldg(reinterpret_cast<const float4*>(rb) + lane + 32 * q);
    }
    float2* z = Z + warp * L1;
#pragma unroll
    for (int q = 0; q < L1 / 128; ++q) {
      const int x = 4 * (lane + 32 * q);
      z[rswz(x)] = make_float2(va[q].x, vb[q].x);
      z[rswz(x + 1)] = make_float2(va[q].y, vb[q].y);
      z[rswz(x + 2)] = make_float2(va[q].z, vb[q].z);
      z[rswz(x + 3)] = make_float2(va[q].w, vb[q].w);
    }
  }
  __syncthreads();
  // 2. forward x FFT; one warp per sequence
  fft_fixed<L1, false, false, L1, 1, -2>(Z, NSEQ, a.tw1, tid, NT);
  // 3. separate the two spectra of each sequence (as ROW_R2C) into the x-spectrum rows
  if (warp < NSEQ) {
    const float2* z = Z + warp * L1;
    float2* A = X + (2 * warp) * XP;
    float2* B = A + XP;
    for (int k = lane; k < NH; k += 32) {
      const float2 zk = z[rswz(k)];
      const float2 zn = z[rswz(k == 0 ? 0 : L1 - k)];
      A[k] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
      B[k] = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
    }
  }
  // 4. every block's x-spectrum rows are complete (and this block's x sequences dead)
  cluster_arrive();
  cluster_wait();
  // 5. gather columns [r*CB, r*CB + nc) of every block's rows into the y tile [L2][W]
  {
    const int k0 = r * CB;
    const int nc = (r == CS - 1) ? CB + 1 : CB;
    constexpr int TOT = CS * RY * W;
    static_assert(TOT % NT == 0 || TOT < NT || true, "");
#pragma unroll 4
    for (int i = tid; i < TOT; i += NT) {
      const int s = i / (RY * W);
      const int rem = i - s * (RY * W);
      const int yl = rem / W, j = rem - yl * W;
      if (j < nc) {
        const float2* Xs = cl.map_shared_rank(X, s);
        Y[(s * RY + yl) * W + j] = Xs[yl * XP + k0 + j];
      }
    }
  }
  // this block has read all it needs from the others
  cluster_arrive();
  __syncthreads();
  // 6. forward y FFT of the tile's columns; the last stage stores to the half spectrum
  {
    ColIO<float2> io;
    io.gin = nullptr;
    io.gout = a.spec + unit * (size_t)L2 * P + (size_t)r * CB;
    io.cstride = 0;
    io.rstride = P;
    io.ccols = W;
    io.ncol = (r == CS - 1) ? CB + 1 : CB;
    fft_col_fixed<L2, W, W, false, false, true>(Y, io, a.tw2, tid, NT);
  }
  // 7. no block leaves while another may still read its x-spectrum rows
  cluster_wait();
}

template <int L1, int L2, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(XYShape<L1, L2, CS>::NT, 2)
    k_xy_inv(const XYArgs a) {
  using S = XYShape<L1, L2, CS>;
  constexpr int NT = S::NT, RY = S::RY, NSEQ = S::NSEQ, W = S::W, XP = S::XP, CB = S::CB;
  constexpr int half = L1 / 2;
  if (a.st->retired || (a.skip_if_done && a.st->done)) return;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* X = reinterpret_cast<float2*>(smraw + S::XOFF);
  float2* Y = reinterpret_cast<float2*>(smraw + S::YOFF);
  float2* Z = reinterpret_cast<float2*>(smraw + S::ZOFF_INV);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = (int)cl.block_rank();
  const size_t unit = blockIdx.x / CS;
  const size_t P = (size_t)a.P;

  // 1. inverse y FFT of columns [r*CB, r*CB + nc); the first stage reads global memory
  {
    ColIO<float2> io;
    io.gin = a.spec + unit * (size_t)L2 * P + (size_t)r * CB;
    io.gout = nullptr;
    io.cstride = 0;
    io.rstride = P;
    io.ccols = (r == CS - 1) ? CB + 1 : CB;
    io.ncol = io.ccols;
    fft_col_fixed<L2, W, W, true, true, false>(Y, io, a.tw2, tid, NT);
  }
  // 2. every block's y tile is complete
  cluster_arrive();
  cluster_wait();
  // 3. gather rows [r*RY, (r+1)*RY) of every block's columns into the x-spectrum rows
  {
    constexpr int TOT = CS * RY * W;
#pragma unroll 4
    for (int i = tid; i < TOT; i += NT) {
      const int s = i / (RY * W);
      const int rem = i - s * (RY * W);
      const int yl = rem / W, j = rem - yl * W;
      const int nc = (s == CS - 1) ? CB + 1 : CB;
      if (j < nc) {
        const float2* Ys = cl.map_shared_rank(Y, s);
        X[yl * XP + s * CB + j] = Ys[(r * RY + yl) * W + j];
      }
    }
  }
  cluster_arrive();
  __syncthreads();
  // 4. Hermitian extension of row pairs (as ROW_C2R), one warp per sequence, then the inverse x FFT
  if (warp < NSEQ) {
    const float2* A = X + (2 * warp) * XP;
    const float2* B = A + XP;
    float2* z = Z + warp * L1;
#pragma unroll 2
    for (int k = lane; k <= half; k += 32) {
      float2 va = A[k], vb = B[k];
      const bool edge = (k == 0 || k == half);
      if (edge) { va.y = 0.f; vb.y = 0.f; }
      z[rswz(k)] = make_float2(va.x - vb.y, va.y + vb.x);
      if (!edge) z[rswz(L1 - k)] = make_float2(va.x + vb.y, vb.x - va.y);
    }
  }
  __syncwarp();
  fft_fixed<L1, true, false, L1, 1, -2>(Z, NSEQ, a.tw1, tid, NT);
  // 5. real rows 2s (real parts) and 2s+1 (imaginary parts)
  if (warp < NSEQ) {
    const float2* z = Z + warp * L1;
    float* ra = a.real_out + (unit * L2 + (size_t)r * RY + 2 * warp) * L1;
    float* rb = ra + L1;
#pragma unroll
    for (int q = 0; q < L1 / 128; ++q) {
      const int x = 4 * (lane + 32 * q);
      const float2 w0 = z[rswz(x)], w1 = z[rswz(x + 1)], w2 = z[rswz(x + 2)], w3 = z[rswz(x + 3)];
      reinterpret_cast<float4*>(ra)[lane + 32 * q] = make_float4(w0.x, w1.x, w2.x, w3.x);
      reinterpret_cast<float4*>(rb)[lane + 32 * q] = make_float4(w0.y, w1.y, w2.y, w3.y);
    }
  }
  // 6. no block leaves while another may still read its y tile
  cluster_wait();
}

}  // namespace hs
