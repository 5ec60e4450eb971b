// Shared device-side definitions of the tetrahedral-stencil solver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace hs {

// Device-resident solve status.  Written by the last block of every
// residual-evaluating kernel (see finalize()); read by every other kernel at
// entry so that the work queued after convergence becomes a no-op.
struct DevStatus {
  int done;       // 0 running, 1 converged, 2 max_iter reached, 3 diverged
  int evals;      // residual evaluations so far
  int max_iter;   // stop (done = 2) after this many evaluations
  int hist_cap;   // capacity of the error history
  unsigned int counter;  // block-arrival counter of the last-block reduction
  int retired;    // batched solves: this item is finished and every kernel skips it
  double tol;       // converged when err < tol
  double err;       // error of the last evaluation, Eq. (tolerance)
  double l2;        // L2 norm of the nodal force, Eq. (L2-norm)
  double sig_norm;  // Frobenius norm of <sigma>
  double sig_mean[6];  // <sigma> = 1/2(<sigma^T1> + <sigma^T2>), Voigt order
  double err_min;
  double denom;     // > 0: use this instead of sig_norm (correction solves)
  double nvox;      // N
  // Applied-stress control (Section 2.5, Algorithm 1 step 6): when macro is
  // not null it points at [sigma^a (6, Voigt), S0 (6x6)], S0 mapping a Voigt
  // stress to the tensor strain components of (lambda0)^-1 : sigma, and every
  // evaluation that does not stop moves the macroscopic strain E (tensor
  // components, read by the kernels of the next evaluation) by
  // S0 (sigma^a - <sigma>).
  const double* macro;
  double E[6];
  // > 0: also converged once err <= rel_tol * (err of the first evaluation of this run)
  double rel_tol;
  double err_first;
};

// DONE_TIMEOUT: a bounded device wait (the mbarrier of a tensor copy) gave up; DONE_FAULT: a
// kernel's own check (the alignment a tensor copy needs) failed before the access.  Both stay set.
enum { DONE_RUNNING = 0, DONE_CONVERGED = 1, DONE_MAXITER = 2, DONE_DIVERGED = 3, DONE_TIMEOUT = 4, DONE_FAULT = 5 };

// Batched launches (one launch over many solves of the same grid): item
// blockIdx.z works in the workspace that starts zstride bytes after item
// blockIdx.z - 1's, so every workspace pointer of the launch moves by
// blockIdx.z * zstride.  zstride = 0: a single solve.
template <typename P> __device__ __forceinline__ P* zshift(P* p, size_t off) {
  return p == nullptr ? p : reinterpret_cast<P*>(reinterpret_cast<uintptr_t>(p) + off);
}
constexpr int NRED = 7;  // sum of sigma^T1 + sigma^T2 (6), sum |F|^2 (1)

// Isotropic phases: per phase (lambda, mu).
template <typename T> struct MatIso {
  const T* tab;
  __device__ __forceinline__ void stress(int ph, const T* e, T* s) const {
    const T lam = __ldg(tab + 2 * ph), mu = __ldg(tab + 2 * ph + 1);
    const T lt = lam * (e[0] + e[1] + e[2]);
    const T m2 = mu + mu;
    s[0] = lt + m2 * e[0];
    s[1] = lt + m2 * e[1];
    s[2] = lt + m2 * e[2];
    s[3] = mu * e[3];
    s[4] = mu * e[4];
    s[5] = mu * e[5];
  }
};

// General anisotropic phases: per phase the 21 upper-triangle entries of the
// 6x6 Voigt stiffness, row-major.  e is the engineering Voigt strain.
template <typename T> struct MatAniso {
  const T* tab;
  __device__ __forceinline__ void stress(int ph, const T* e, T* s) const {
    const T* c = tab + 21 * ph;
    T C[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) C[i] = __ldg(c + i);
    // index of (i,j), i <= j, in the packed upper triangle
#define HS_UT(i, j) ((i) * 6 - ((i) * ((i) - 1)) / 2 + ((j) - (i)))
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < 6; ++j) acc += C[i <= j ? HS_UT(i, j) : HS_UT(j, i)] * e[j];
      s[i] = acc;
    }
#undef HS_UT
  }
};

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Evaluation of the stopping test from the sums of one residual evaluation
// (Eqs. L2-norm, tolerance): sums[0..5] = sum over voxels of sigma^T1 + sigma^T2,
// sums[6] = sum over corners of |F|^2.  Updates the status (error, history,
// done flag, applied-stress strain update) and clears the arrival counter.
// One thread calls it.
__device__ inline void finalize_eval(DevStatus* st, double* hist, const double* sums) {
  if (st->done == DONE_TIMEOUT || st->done == DONE_FAULT) {
    st->counter = 0;
    return;
  }
  const double n = st->nvox;
  double sm[6], nrm2 = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    sm[i] = 0.5 * sums[i] / n;
    nrm2 += (i < 3 ? 1.0 : 2.0) * sm[i] * sm[i];
    st->sig_mean[i] = sm[i];
  }
  const double l2 = sqrt(sums[6] / n);
  const double nrm = sqrt(nrm2);
  const double den = st->denom > 0 ? st->denom : nrm;
  double err;
  if (den > 0) err = l2 / den;
  else err = (l2 == 0) ? 0.0 : __longlong_as_double(0x7ff0000000000000LL);
  st->l2 = l2;
  st->sig_norm = nrm;
  st->err = err;
  const int k = st->evals;
  if (k < st->hist_cap) hist[k] = err;
  st->evals = k + 1;
  if (!(err == err) || err > 1e300) {
    st->done = DONE_DIVERGED;
  } else {
    if (k == 0 || err < st->err_min) st->err_min = err;
    if (k == 0) st->err_first = err;
    if (err < st->tol || (st->rel_tol > 0 && err <= st->rel_tol * st->err_first)) st->done = DONE_CONVERGED;
    else if (err > 1e6 * st->err_min && k > 10) st->done = DONE_DIVERGED;
    else if (k + 1 >= st->max_iter) st->done = DONE_MAXITER;
  }
  if (st->macro != nullptr && st->done == DONE_RUNNING) {
    // E <- (lambda0)^-1 : {sigma^a + (lambda0 - <lambda>) : E - <lambda : deps> + <lambda : eps0>}
    //    = E + (lambda0)^-1 : (sigma^a - <sigma>)   (the same quantity, regrouped)
    const double* Sa = st->macro;
    const double* S0 = st->macro + 6;
    double d[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = Sa[i] - sm[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double acc = 0;
#pragma unroll
      for (int j = 0; j < 6; ++j) acc += S0[i * 6 + j] * d[j];
      st->E[i] += acc;
    }
  }
  st->counter = 0;
}

// Block-sum NV doubles (fixed order) into dst[0 .. NV-1].  scratch: >= 32 * NV
// doubles of shared memory.  Every thread of the block must call it.
template <int NV>
__device__ inline void block_sum(const double (&acc)[NV], double* dst, double* scratch) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = warp_sum(acc[v]);
    if (lane == 0) scratch[warp * NV + v] = s;
  }
  __syncthreads();
  if (tid < NV) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += scratch[w * NV + tid];
    dst[tid] = s;
  }
}

// After every block has written its partials: true in the one block that
// arrives last (all partials of the launch visible to it).
__device__ inline bool last_block_arrived(DevStatus* st, unsigned int nblk) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(&st->counter, 1u);
    am_last = (prev == nblk - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Block-sum NRED doubles (fixed order) and publish them as this block's
// partials; the last block to arrive reduces all partials in index order and
// evaluates the stopping test.  scratch: >= 32 * NRED doubles of shared memory.
__device__ inline void reduce_and_finalize(const double (&acc)[NRED], double* partials, DevStatus* st,
                                           double* hist, double* scratch) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
  const int nblk = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  block_sum<NRED>(acc, partials + (size_t)bid * NRED, scratch);
  if (!last_block_arrived(st, (unsigned)nblk)) return;
  // deterministic: value v by warp (v mod nw), lanes stride over blocks
  for (int v = warp; v < NRED; v += nw) {
    double s = 0;
    for (int b = lane; b < nblk; b += 32) s += __ldcg(partials + (size_t)b * NRED + v);
    s = warp_sum(s);
    if (lane == 0) scratch[v] = s;
  }
  __syncthreads();
  if (tid == 0) finalize_eval(st, hist, scratch);
}

// ---- mbarriers and tensor (TMA) copies ------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the async proxy (then a block barrier)
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Wait for the completion of the barrier phase of the given parity, at most about 2^22 tries
// (each try may suspend the thread for a while); false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const uint32_t b = smem_u32(bar);
  for (int i = 0; i < (1 << 22); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// Tiled tensor copy global -> shared of the box at coordinates (c0 .. c4) of a rank-5 tensor map
// (a __grid_constant__ kernel parameter), completing on the mbarrier.  The innermost coordinate
// times the element size must be a multiple of 16 bytes; dst 128-byte aligned.
__device__ __forceinline__ void tma_load_5d(void* dst, const void* tmap, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace hs
