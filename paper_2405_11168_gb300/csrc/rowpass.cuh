// Row passes: FFTs along x between real rows and the half spectrum.
//
// ROW_C2R: two half-spectrum rows A, B (N1/2 + 1 complex values each) become
//   the complex sequence Z[k] = A[k] + i B[k] (k <= N1/2, imaginary parts of
//   the k = 0 and k = N1/2 bins dropped) extended by Z[N1-k] = conj(A[k]) +
//   i conj(B[k]); its unnormalised inverse FFT gives the two real rows as
//   Re Z and Im Z.
// ROW_R2C: two real rows a, b form Z = a + i b; after the forward FFT
//   A[k] = (Z[k] + conj Z[N1-k]) / 2 and B[k] = (Z[k] - conj Z[N1-k]) / (2i).
//
// A group of T = N1/8 threads owns one pair of rows at a time; for N1 <= 256
// the group lies inside one warp and needs only warp barriers.
#pragma once
#include "common.cuh"

namespace hs {

enum { ROW_C2R = 0, ROW_R2C = 1 };

template <typename T> struct RowArgs {
  using C = typename cplx_t<T>::type;
  const C* spec_in;   // C2R: half-spectrum rows [nrows][P]
  C* spec_out;        // R2C
  const T* real_in;   // R2C: real rows [nrows][n1]
  T* real_out;        // C2R
  double* acc64;      // C2R optional: acc64[row][x] += real value (FP64 accumulation)
  const C* tw;        // w_N1^j
  FftPlan plan;
  int n1, P, nrows;
  const DevStatus* st;
  int skip_if_done;
};

__device__ __forceinline__ void group_sync(bool wsync) {
  if (wsync) __syncwarp();
  else __syncthreads();
}

// LF > 0: N1 = LF and 256 threads per block, fixed at compile time (hot
// sizes); LF = 0: both taken at run time.
template <typename T, int MODE, int LF = 0>
__global__ void __launch_bounds__(256, 3) k_row(const RowArgs<T> a) {
  using C = typename cplx_t<T>::type;
  if (a.skip_if_done && a.st->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n1 = LF > 0 ? LF : a.n1, P = a.P, nh = n1 / 2 + 1, half = n1 / 2;
  const int tid = threadIdx.x, nthr = LF > 0 ? 256 : (int)blockDim.x;
  const int T8 = (n1 + kE - 1) / kE;          // threads per sequence
  const int G = nthr / T8;                     // sequences per block pass
  const int grp = tid / T8, t = tid - grp * T8;
  const bool wsync = T8 <= 32 && (32 % T8) == 0;
  const int pitch = rpitch(n1);
  C* z = reinterpret_cast<C*>(smraw) + (size_t)grp * pitch;
  const int nseq = a.nrows / 2;
  const FftPlan plan = a.plan;
  for (int s0 = blockIdx.x * G; s0 < nseq; s0 += gridDim.x * G) {
    const int s = s0 + grp;
    const bool act = grp < G && s < nseq;
    const size_t r0 = 2 * (size_t)s, r1 = r0 + 1;
    if (MODE == ROW_C2R) {
      if (act) {
        const C* A = a.spec_in + r0 * P;
        const C* B = a.spec_in + r1 * P;
#pragma unroll 4
        for (int k = t; k < n1; k += T8) {
          const int kk = (k <= half) ? k : n1 - k;
          C va = A[kk], vb = B[kk];
          if (kk == 0 || kk == half) { va.y = 0; vb.y = 0; }
          C w;
          if (k <= half) { w.x = va.x - vb.y; w.y = va.y + vb.x; }
          else { w.x = va.x + vb.y; w.y = vb.x - va.y; }
          z[rpad(k)] = w;
        }
      }
      group_sync(wsync);
      if constexpr (LF > 0) {
        fft_fixed<LF, true, false, LF + LF / 8 + 1, 1, 3>(reinterpret_cast<C*>(smraw), G, a.tw, tid, nthr);
      } else {
        fft_smem<true, false>(reinterpret_cast<C*>(smraw), pitch, 1, 3, G, plan.L, plan.nstage, plan.packed, a.tw,
                              tid, nthr);
      }
      group_sync(wsync);
      if (act) {
        for (int x = t; x < n1; x += T8) {
          const C w = z[rpad(x)];
          if (a.real_out) {
            a.real_out[r0 * n1 + x] = w.x;
            a.real_out[r1 * n1 + x] = w.y;
          }
          if (a.acc64) {
            a.acc64[r0 * n1 + x] += (double)w.x;
            a.acc64[r1 * n1 + x] += (double)w.y;
          }
        }
      }
    } else {
      if (act) {
        const T* ra = a.real_in + r0 * n1;
        const T* rb = a.real_in + r1 * n1;
#pragma unroll 4
        for (int x = t; x < n1; x += T8) {
          C w;
          w.x = ra[x];
          w.y = rb[x];
          z[rpad(x)] = w;
        }
      }
      group_sync(wsync);
      if constexpr (LF > 0) {
        fft_fixed<LF, false, false, LF + LF / 8 + 1, 1, 3>(reinterpret_cast<C*>(smraw), G, a.tw, tid, nthr);
      } else {
        fft_smem<false, false>(reinterpret_cast<C*>(smraw), pitch, 1, 3, G, plan.L, plan.nstage, plan.packed, a.tw,
                              tid, nthr);
      }
      group_sync(wsync);
      if (act) {
        C* A = a.spec_out + r0 * P;
        C* B = a.spec_out + r1 * P;
        for (int k = t; k < nh; k += T8) {
          const C zk = z[rpad(k)];
          const C zn = z[rpad(k == 0 ? 0 : n1 - k)];
          C va, vb;
          va.x = T(0.5) * (zk.x + zn.x);
          va.y = T(0.5) * (zk.y - zn.y);
          vb.x = T(0.5) * (zk.y + zn.y);
          vb.y = T(0.5) * (zn.x - zk.x);
          A[k] = va;
          B[k] = vb;
        }
      }
    }
    group_sync(wsync);
  }
}

}  // namespace hs
