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
// the group lies inside one warp and needs only warp barriers.  Blocks are
// persistent and stage their next batch of input rows with cp.async while
// transforming the current one.
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
  DevStatus* st;
  int skip_if_done;
  size_t zstride;     // batched launches: bytes between the workspaces of consecutive items
};

template <typename T> __device__ __forceinline__ RowArgs<T> row_item_args(const RowArgs<T>& a) {
  if (a.zstride == 0) return a;
  RowArgs<T> b = a;
  const size_t o = (size_t)blockIdx.z * a.zstride;
  b.spec_in = zshift(a.spec_in, o);
  b.spec_out = zshift(a.spec_out, o);
  b.real_in = zshift(a.real_in, o);
  b.real_out = zshift(a.real_out, o);
  b.acc64 = zshift(a.acc64, o);
  b.tw = zshift(a.tw, o);
  b.st = zshift(a.st, o);
  return b;
}

__device__ __forceinline__ void group_sync(bool wsync) {
  if (wsync) __syncwarp();
  else __syncthreads();
}

// Shared memory of k_row: FFT rows z[G][rpitch(n1)], then two staging buffers
// of one batch (2G rows) each; a staging buffer holds the batch's input rows,
// then (bulk-store path) its output rows.  Host and device use the same function.
struct RowLayout {
  int G;            // sequences (row pairs) per batch
  size_t zbytes;    // z rows
  size_t rowbytes;  // bytes of one input row (C2R: P complex; R2C: n1 real)
  size_t outbytes;  // bytes of one output row (C2R: n1 real; R2C: P complex)
  size_t stage;     // bytes of one staging buffer
  size_t bar;       // two mbarriers of the staging buffers (bulk-copy loads)
  size_t tws;       // the per-stage twiddle table (fewer than n1 complex values; fixed lengths)
  size_t total;
};
__host__ __device__ inline RowLayout row_layout(int mode, int n1, int P, int nthr, int tsize) {
  RowLayout L;
  const int T8 = (n1 + kE - 1) / kE;
  L.G = nthr / T8;
  L.zbytes = (((size_t)L.G * rpitch(n1) * 2 * tsize) + 15) & ~(size_t)15;
  L.rowbytes = (mode == ROW_C2R) ? (size_t)P * 2 * tsize : (size_t)n1 * tsize;
  L.outbytes = (mode == ROW_C2R) ? (size_t)n1 * tsize : (size_t)P * 2 * tsize;
  const size_t rb = L.rowbytes > L.outbytes ? L.rowbytes : L.outbytes;
  L.stage = ((2 * (size_t)L.G * rb) + 15) & ~(size_t)15;
  L.bar = L.zbytes + 2 * L.stage;
  L.tws = L.bar + 16;
  L.total = L.tws + (size_t)n1 * 2 * tsize;
  return L;
}

// Asynchronous copy of batch b (input rows 2bG .. 2bG + 2G - 1, clipped to
// nrows) into staging buffer `buf`: the rows are one contiguous byte range.
// bulk: one cp.async.bulk by the calling thread, completing on the buffer's
// mbarrier (rows of a multiple of 16 bytes); otherwise 16-byte cp.async by
// every thread and a commit.
template <typename T, int MODE>
__device__ __forceinline__ void row_stage(const RowArgs<T>& a, const RowLayout& L, unsigned char* smraw, int b,
                                          int buf, bool bulk = false) {
  const size_t r0 = 2 * (size_t)b * L.G;
  const size_t nr = min((size_t)2 * L.G, (size_t)a.nrows - r0);
  const unsigned char* src = (MODE == ROW_C2R) ? reinterpret_cast<const unsigned char*>(a.spec_in)
                                               : reinterpret_cast<const unsigned char*>(a.real_in);
  src += r0 * L.rowbytes;
  unsigned char* dst = smraw + L.zbytes + (size_t)buf * L.stage;
  const size_t bytes = nr * L.rowbytes;
  if (bulk) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + L.bar) + buf;
    mbar_arrive_expect_tx(bar, (unsigned)bytes);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"((unsigned)bytes), "r"(smem_u32(bar))
                 : "memory");
    return;
  }
  if ((L.rowbytes & 15) == 0) {
    const int nch = (int)(bytes >> 4);
    for (int i = threadIdx.x; i < nch; i += blockDim.x) cp_async16(dst + 16 * i, src + 16 * i);
  } else {
    // rows of a size that is not a multiple of 16 bytes (R2C with N1 % 4 != 0): element copies
    const T* s = reinterpret_cast<const T*>(src);
    T* d = reinterpret_cast<T*>(dst);
    for (size_t i = threadIdx.x; i < bytes / sizeof(T); i += blockDim.x) d[i] = s[i];
  }
  cp_async_commit();
}

// Persistent: block j transforms batches j, j + gridDim.x, ...; the copy of the
// next batch runs while the current one is transformed.
// LF > 0: N1 = LF and 256 threads per block, fixed at compile time (hot
// sizes); LF = 0: both taken at run time; LF = -1: run time, plans with a
// radix-5, 7 or 11 stage.
// BATCH: a batched launch (grid.z items); a single solve's launch uses the arguments as they come.
template <typename T, int MODE, int LF = 0, bool BATCH = false>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 3) k_row(const RowArgs<T> a_) {
  using C = typename cplx_t<T>::type;
  const RowArgs<T> a = BATCH ? row_item_args(a_) : a_;
  if (a.st->retired || (a.skip_if_done && a.st->done)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n1 = LF > 0 ? LF : a.n1, P = a.P, nh = n1 / 2 + 1, half = n1 / 2;
  const int tid = threadIdx.x, nthr = LF > 0 ? 256 : (int)blockDim.x;
  const RowLayout L = row_layout(MODE, n1, P, nthr, (int)sizeof(T));
  const int T8 = (n1 + kE - 1) / kE;          // threads per sequence
  const int G = L.G;                           // sequences per batch
  const int grp = tid / T8, t = tid - grp * T8;
  const bool wsync = T8 <= 32 && (32 % T8) == 0;
  // fixed lengths: XOR-swizzled rows (length-64 rows 72 apart, so that the
  // four rows a warp transforms fall on different banks); otherwise one spare
  // slot per 8
  constexpr int FP = LF == 64 ? 72 : (LF > 0 ? LF : 1);
  const int pitch = LF > 0 ? FP : rpitch(n1);
  C* z = reinterpret_cast<C*>(smraw) + (size_t)grp * pitch;
  auto zi = [](int e) { return LF > 0 ? rswz(e) : rpad(e); };
  // fixed lengths: the positions of elements t + j T8 and n1 - (t + j T8) from the thread's
  // swizzled offsets and one XOR with a constant (the swizzle is linear over XOR; see fft.cuh)
  constexpr int T8C = LF > 0 ? LF / kE : 1;
  const int tsw = LF > 0 ? rswz(t) : 0;
  const int tmir = (LF > 0 && t > 0) ? rswz(T8C - t) : 0;
  auto zfwd = [&](int j) { return LF > 0 ? (tsw ^ swz_c(j * T8C)) : zi(t + j * T8); };
  auto zmir = [&](int j) {  // position of n1 - (t + j T8), for t + j T8 > 0
    if (LF > 0) return t == 0 ? swz_c(LF - j * T8C) : (tmir ^ swz_c(LF - (j + 1) * T8C));
    return zi(n1 - t - j * T8);
  };
  const int nseq = a.nrows / 2;
  const int nbatch = (nseq + G - 1) / G;
  const FftPlan plan = a.plan;
  // fixed lengths, C2R: a batch's real output rows are assembled in its staging
  // buffer and written by one bulk copy (FP64 accumulation keeps per-element
  // updates).  R2C measured faster with direct stores (0.104 vs 0.112 ms at 256^3).
  const bool bulk = LF > 0 && MODE == ROW_C2R && a.acc64 == nullptr && (L.outbytes & 15) == 0;
  // fixed lengths: each batch arrives by one bulk copy on its staging buffer's mbarrier (waits
  // bounded; a timeout is recorded in the status)
  const bool bload = LF > 0 && (L.rowbytes & 15) == 0;
  uint64_t* sbar = reinterpret_cast<uint64_t*>(smraw + L.bar);
  bool timed_out = false;
  if (bload) {
    if (tid == 0) {
      mbar_init(sbar, 1);
      mbar_init(sbar + 1, 1);
      mbar_init_fence();
    }
    __syncthreads();
  }
  // fixed lengths: the transforms read their twiddles from the plan's per-stage table in shared
  // memory (first read after the barrier that opens the first batch)
  C* const tws = reinterpret_cast<C*>(smraw + L.tws);
  if constexpr (LF > 0) stage_twiddles<LF>(tws, a.tw, tid, nthr);
  int buf = 0;
  if ((int)blockIdx.x < nbatch && (!bload || tid == 0)) row_stage<T, MODE>(a, L, smraw, blockIdx.x, 0, bload);
  int k = 0;
  for (int b = blockIdx.x; b < nbatch; b += gridDim.x, buf ^= 1, ++k) {
    if (bload) timed_out |= !mbar_wait(sbar + buf, (unsigned)((k >> 1) & 1));
    else cp_async_wait_all();
    if (bulk && tid == 0) bulk_wait_read_all();  // staging buffer buf ^ 1 is free again
    __syncthreads();
    if (b + (int)gridDim.x < nbatch && (!bload || tid == 0))
      row_stage<T, MODE>(a, L, smraw, b + gridDim.x, buf ^ 1, bload);
    unsigned char* stg = smraw + L.zbytes + (size_t)buf * L.stage;
    const size_t nr = min((size_t)2 * G, (size_t)a.nrows - 2 * (size_t)b * G);
    const int s = b * G + grp;
    const bool act = grp < G && s < nseq;
    const size_t r0 = 2 * (size_t)s, r1 = r0 + 1;
    if (MODE == ROW_C2R) {
      if (act) {
        const C* A = reinterpret_cast<const C*>(stg + (size_t)(2 * grp) * L.rowbytes);
        const C* B = reinterpret_cast<const C*>(stg + (size_t)(2 * grp + 1) * L.rowbytes);
        // Z[k] and its mirror Z[N1-k] from one read of A[k], B[k]
        if constexpr (LF > 0) {
#pragma unroll
          for (int j = 0; j <= LF / 2 / T8C; ++j) {
            const int k = t + j * T8C;
            if (k <= half) {
              C va = A[k], vb = B[k];
              const bool edge = (k == 0 || k == half);
              if (edge) { va.y = 0; vb.y = 0; }
              z[zfwd(j)] = cmk<C>(va.x - vb.y, va.y + vb.x);
              if (!edge) z[zmir(j)] = cmk<C>(va.x + vb.y, vb.x - va.y);
            }
          }
        } else {
#pragma unroll 2
          for (int k = t; k <= half; k += T8) {
            C va = A[k], vb = B[k];
            const bool edge = (k == 0 || k == half);
            if (edge) { va.y = 0; vb.y = 0; }
            z[zi(k)] = cmk<C>(va.x - vb.y, va.y + vb.x);
            if (!edge) z[zi(n1 - k)] = cmk<C>(va.x + vb.y, vb.x - va.y);
          }
        }
      }
      group_sync(wsync);
      if constexpr (LF > 0) {
        fft_fixed<LF, true, false, FP, 1, -2, true>(reinterpret_cast<C*>(smraw), G, tws, tid, nthr);
      } else {
        fft_smem<true, false, (LF < 0)>(reinterpret_cast<C*>(smraw), pitch, 1, 3, G, plan.L, plan.nstage, plan.packed, a.tw,
                              tid, nthr);
      }
      if (bulk) {
        __syncthreads();  // every group is done with the staged input
        if (act) {
          T* o = reinterpret_cast<T*>(stg) + (size_t)(2 * grp) * n1;
          if constexpr (LF > 0) {
#pragma unroll
            for (int j = 0; j < LF / T8C; ++j) {
              const C w = z[zfwd(j)];
              o[t + j * T8C] = w.x;
              o[n1 + t + j * T8C] = w.y;
            }
          } else {
            for (int x = t; x < n1; x += T8) {
              const C w = z[zi(x)];
              o[x] = w.x;
              o[n1 + x] = w.y;
            }
          }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
          bulk_s2g(a.real_out + 2 * (size_t)b * G * n1, stg, (unsigned)(nr * L.outbytes));
          bulk_commit();
        }
        continue;
      }
      group_sync(wsync);
      if (act) {
        for (int x = t; x < n1; x += T8) {
          const C w = z[zi(x)];
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
        const T* ra = reinterpret_cast<const T*>(stg + (size_t)(2 * grp) * L.rowbytes);
        const T* rb = reinterpret_cast<const T*>(stg + (size_t)(2 * grp + 1) * L.rowbytes);
        if constexpr (LF > 0) {
#pragma unroll
          for (int j = 0; j < LF / T8C; ++j) {
            C w;
            w.x = ra[t + j * T8C];
            w.y = rb[t + j * T8C];
            z[zfwd(j)] = w;
          }
        } else {
#pragma unroll 4
          for (int x = t; x < n1; x += T8) {
            C w;
            w.x = ra[x];
            w.y = rb[x];
            z[zi(x)] = w;
          }
        }
      }
      group_sync(wsync);
      if constexpr (LF > 0) {
        fft_fixed<LF, false, false, FP, 1, -2, true>(reinterpret_cast<C*>(smraw), G, tws, tid, nthr);
      } else {
        fft_smem<false, false, (LF < 0)>(reinterpret_cast<C*>(smraw), pitch, 1, 3, G, plan.L, plan.nstage, plan.packed, a.tw,
                               tid, nthr);
      }
      if (bulk) {
        __syncthreads();  // every group is done with the staged input
        if (act) {
          C* A = reinterpret_cast<C*>(stg) + (size_t)(2 * grp) * P;
          C* B = A + P;
          for (int k = t; k < P; k += T8) {
            C va = cmk<C>(0, 0), vb = cmk<C>(0, 0);
            if (k < nh) {
              const C zk = z[zi(k)];
              const C zn = z[zi(k == 0 ? 0 : n1 - k)];
              va = cmk<C>(T(0.5) * (zk.x + zn.x), T(0.5) * (zk.y - zn.y));
              vb = cmk<C>(T(0.5) * (zk.y + zn.y), T(0.5) * (zn.x - zk.x));
            }
            A[k] = va;
            B[k] = vb;
          }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
          bulk_s2g(a.spec_out + 2 * (size_t)b * G * P, stg, (unsigned)(nr * L.outbytes));
          bulk_commit();
        }
        continue;
      }
      group_sync(wsync);
      if (act) {
        C* A = a.spec_out + r0 * P;
        C* B = a.spec_out + r1 * P;
        // A[k], B[k] from Z[k] and Z[N1-k] (k = 0: Z[0] twice)
        auto separate = [&](int k, const C zk, const C zn) {
          C va, vb;
          va.x = T(0.5) * (zk.x + zn.x);
          va.y = T(0.5) * (zk.y - zn.y);
          vb.x = T(0.5) * (zk.y + zn.y);
          vb.y = T(0.5) * (zn.x - zk.x);
          A[k] = va;
          B[k] = vb;
        };
        if constexpr (LF > 0) {
#pragma unroll
          for (int j = 0; j <= LF / 2 / T8C; ++j) {
            const int k = t + j * T8C;
            if (k < nh) separate(k, z[zfwd(j)], z[k == 0 ? 0 : zmir(j)]);
          }
        } else {
          for (int k = t; k < nh; k += T8) separate(k, z[zi(k)], z[zi(k == 0 ? 0 : n1 - k)]);
        }
      }
    }
  }
  cp_async_wait_all();
  if (bulk && tid == 0) bulk_wait_all();
  if (timed_out) a.st->done = DONE_TIMEOUT;
}

}  // namespace hs
