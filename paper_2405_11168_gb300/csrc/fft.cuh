// Batched mixed-radix (2/3/4/8/16, and 5/7/11) complex FFTs on sequences held in shared memory.
//
// Self-sorting Stockham formulation, one radix-R butterfly per (thread, step):
// stage s with radix R and Ns = R_1...R_{s-1} reads x[b + m L/R], multiplies by
// the twiddle w_{Ns R}^{(b mod Ns) m}, takes a length-R DFT and writes
// y[(b div Ns) Ns R + (b mod Ns) + m Ns].  After the last stage the result is in
// natural order.  Every stage is done in place: a thread loads all of its
// butterflies' inputs into registers, the block synchronises, then it writes.
//
// Threads per sequence: ceil(L/kE) with kE = 8 elements per thread, so a
// thread never holds more than ceil(kE/R) butterflies of one stage; radices
// are 8, 4, 3 and 2 (a radix-16 DFT is available but keeps too many values
// live for the generic stage loop), and 5, 7 and 11 for the other supported
// lengths: their length-R DFT is the plain O(R^2) sum with coefficients
// w_R^{mk} = w_L^{(L/R)(mk mod R)} read from the same twiddle table.  Sequence s, element e lives at
// buf[s*ss + e*es].  Forward = exp(-2 pi i nk/L), inverse = exp(+...), both
// unnormalised.  Twiddles come from a per-axis table w_L^j = exp(-2 pi i j/L),
// j < L, computed on the host.
#pragma once
#include <cuda_runtime.h>

namespace hs {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
// multiply by -i (forward quarter turn) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a) {
  return INV ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

// cos and sin of 2 pi J / 16 (exact constants of the regular 16-gon)
#define HS_FFT_C1 0.92387953251128675613
#define HS_FFT_S1 0.38268343236508977173
#define HS_FFT_H 0.70710678118654752440
__host__ __device__ constexpr double cos16c(int j) {
  return ((j & 15) == 0) ? 1.0 : ((j & 15) == 1) ? HS_FFT_C1 : ((j & 15) == 2) ? HS_FFT_H : ((j & 15) == 3) ? HS_FFT_S1
       : ((j & 15) == 4) ? 0.0 : ((j & 15) == 5) ? -HS_FFT_S1 : ((j & 15) == 6) ? -HS_FFT_H : ((j & 15) == 7) ? -HS_FFT_C1
       : ((j & 15) == 8) ? -1.0 : ((j & 15) == 9) ? -HS_FFT_C1 : ((j & 15) == 10) ? -HS_FFT_H : ((j & 15) == 11) ? -HS_FFT_S1
       : ((j & 15) == 12) ? 0.0 : ((j & 15) == 13) ? HS_FFT_S1 : ((j & 15) == 14) ? HS_FFT_H : HS_FFT_C1;
}
// sin(t) = cos(t + 3 pi / 2)
__host__ __device__ constexpr double sin16c(int j) { return cos16c(j + 12); }
// w16^J for the requested direction (forward: exp(-2 pi i J/16))
template <int J, bool INV, typename C> __device__ __forceinline__ C w16() {
  using R = decltype(C::x);
  constexpr double c = cos16c(J), sn = sin16c(J);
  return cmk<C>((R)c, INV ? (R)sn : (R)-sn);
}

template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<2, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV, typename C> struct Dft<3, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    using R = decltype(C::x);
    const R h = (R)0.86602540378443864676;  // sqrt(3)/2
    C s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C x0 = v[0];
    C m = cmk<C>(x0.x - (R)0.5 * s.x, x0.y - (R)0.5 * s.y);
    // forward: X1 = m - i h d, X2 = m + i h d
    C ihd = cmk<C>(-h * d.y, h * d.x);  // i h d
    v[0] = cadd(x0, s);
    if (INV) {
      v[1] = cadd(m, ihd);
      v[2] = csub(m, ihd);
    } else {
      v[1] = csub(m, ihd);
      v[2] = cadd(m, ihd);
    }
  }
};

template <bool INV, typename C> struct Dft<4, INV, C> {
  static __device__ __forceinline__ void run(C* v) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

// composite DFT of length A*B: n = B n1 + n2, k = k1 + A k2
template <int A, int B, bool INV, typename C, int N2 = 1, int K1 = 1>
__device__ __forceinline__ void twiddle_all(C (&y)[B][A]) {
  if constexpr (N2 < B) {
    if constexpr (K1 < A) {
      y[N2][K1] = cmul(y[N2][K1], w16<(16 / (A * B)) * N2 * K1, INV, C>());
      twiddle_all<A, B, INV, C, N2, K1 + 1>(y);
    } else {
      twiddle_all<A, B, INV, C, N2 + 1, 1>(y);
    }
  }
}

template <int A, int B, bool INV, typename C> __device__ __forceinline__ void dft_composite(C* v) {
  C y[B][A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) y[n2][n1] = v[B * n1 + n2];
    Dft<A, INV, C>::run(y[n2]);
  }
  twiddle_all<A, B, INV, C>(y);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    C z[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) z[n2] = y[n2][k1];
    Dft<B, INV, C>::run(z);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = z[k2];
  }
}

template <bool INV, typename C> struct Dft<8, INV, C> {
  static __device__ __forceinline__ void run(C* v) { dft_composite<2, 4, INV>(v); }
};
template <bool INV, typename C> struct Dft<16, INV, C> {
  static __device__ __forceinline__ void run(C* v) { dft_composite<4, 4, INV>(v); }
};

// 16-byte asynchronous global -> shared copies (cp.async, bypassing L1).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Bulk shared -> global copies (cp.async.bulk, bulk-group completion).  Both
// addresses 16-byte aligned, size a multiple of 16.  The writes that filled
// the shared source must be made visible to the async proxy first
// (fence_async_smem() by every writing thread, then a barrier).
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, unsigned bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(ssrc));
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(s), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the shared sources of all committed bulk copies may be overwritten
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// all committed bulk copies are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

constexpr int kMaxStages = 8;
// Radix of each stage packed 4 bits per stage (stage 0 in the low bits), so
// the plan is three plain integers and never needs indexed storage.
struct FftPlan {
  int L;       // sequence length
  int nstage;  // number of radix stages (<= kMaxStages)
  int packed;  // radix of stage s = (packed >> 4 s) & 15, product = L
};

// One Stockham stage over the sequences handled by this thread.
constexpr int kE = 8;

template <int R, bool INV, typename C>
__device__ __forceinline__ void stockham_stage(C* buf, int ss, int es, int ps, int s, int t, int T, bool active,
                                               int L, int Ns, int nsh, const C* __restrict__ tw, bool wsync) {
  // element e of sequence s lives at buf[s*ss + e*es + (ps >= 0 ? e >> ps : 0)]
  // nsh >= 0: Ns = 2^nsh (shift/mask index math), else generic division
  constexpr int KB = (kE + R - 1) / R;
  C v[KB][R];
  const int nb = L / R;
  const int step = L / (Ns * R);
  C* sb = buf + s * ss;
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int b = t + k * T;
    if (active && b < nb) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int e = b + m * nb;
        v[k][m] = sb[e * es + (ps >= 0 ? (e >> ps) : 0)];
      }
    }
  }
  if (wsync) __syncwarp(); else __syncthreads();
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int b = t + k * T;
    if (active && b < nb) {
      const int kk = (nsh >= 0) ? (b & (Ns - 1)) : (b % Ns);
      const int pq = (nsh >= 0) ? (b >> nsh) : (b / Ns);
      if (Ns > 1) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          C w = __ldg(tw + kk * m * step);
          if (INV) w.y = -w.y;
          v[k][m] = cmul(v[k][m], w);
        }
      }
      const int base = pq * Ns * R + kk;
      if constexpr (R == 5 || R == 7 || R == 11) {
        // table DFT: each output straight to its place (no array of R outputs kept live)
        const int tstep = L / R;
#pragma unroll 1
        for (int q = 0; q < R; ++q) {
          C acc = v[k][0];
#pragma unroll
          for (int m = 1; m < R; ++m) {
            C w = __ldg(tw + tstep * ((m * q) % R));
            if (INV) w.y = -w.y;
            acc = cadd(acc, cmul(v[k][m], w));
          }
          const int e = base + q * Ns;
          sb[e * es + (ps >= 0 ? (e >> ps) : 0)] = acc;
        }
      } else {
        Dft<R, INV, C>::run(v[k]);
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const int e = base + m * Ns;
          sb[e * es + (ps >= 0 ? (e >> ps) : 0)] = v[k][m];
        }
      }
    }
  }
  if (wsync) __syncwarp(); else __syncthreads();
}

// FFT of nseq sequences in place.  All threads of the block must call this.
// T = ceil(L/kE) threads per sequence, G = blockDim / T sequences per group.
// COLMAP = false: thread i works on sequence g0 + i / T (lanes walk along one
// sequence: for sequences stored as rows, element stride es = 1, padded with
// ps = 3, i.e. one spare slot per 8 elements).  COLMAP = true: thread i works
// on sequence g0 + i % G (lanes walk across sequences: for column tiles whose
// sequences are adjacent in memory, ss = 1).  Either way a warp's shared-memory
// accesses stay (nearly) free of bank conflicts.
// EXT: also radices 5, 7, 11 (their stages keep more values live, so only the
// kernels instantiated for such lengths carry them).
template <bool INV, bool COLMAP, bool EXT = false, typename C>
__device__ __forceinline__ void fft_smem(C* buf, int ss, int es, int ps, int nseq, int L, int nstage, int packed,
                                         const C* __restrict__ tw, int tid, int nthreads) {
  const int T = (L + kE - 1) / kE;
  const int G = nthreads / T;
  for (int g0 = 0; g0 < nseq; g0 += G) {
    const int sl = COLMAP ? (tid % G) : (tid / T);
    const int t = COLMAP ? (tid / G) : (tid % T);
    const int s = g0 + sl;
    const bool active = (COLMAP ? (t < T) : (sl < G)) && s < nseq;
    // row mapping with T dividing 32: every sequence lives inside one warp,
    // so a warp barrier orders its stages (the caller syncs the block after)
    const bool wsync = !COLMAP && T <= 32 && (32 % T) == 0 && (nthreads % 32) == 0;
    int Ns = 1, nsh = 0;
#pragma unroll 1
    for (int st = 0; st < nstage; ++st) {
      const int R = (packed >> (4 * st)) & 15;
      if (R == 8) stockham_stage<8, INV>(buf, ss, es, ps, s, t, T, active, L, Ns, nsh, tw, wsync);
      else if (R == 4) stockham_stage<4, INV>(buf, ss, es, ps, s, t, T, active, L, Ns, nsh, tw, wsync);
      else if (R == 3) stockham_stage<3, INV>(buf, ss, es, ps, s, t, T, active, L, Ns, nsh, tw, wsync);
      else if (EXT && R == 5) stockham_stage<EXT ? 5 : 2, INV>(buf, ss, es, ps, s, t, T, active, L, Ns, nsh, tw, wsync);
      else if (EXT && R == 7) stockham_stage<EXT ? 7 : 2, INV>(buf, ss, es, ps, s, t, T, active, L, Ns, nsh, tw, wsync);
      else if (EXT && R == 11) stockham_stage<EXT ? 11 : 2, INV>(buf, ss, es, ps, s, t, T, active, L, Ns, nsh, tw, wsync);
      else stockham_stage<2, INV>(buf, ss, es, ps, s, t, T, active, L, Ns, nsh, tw, wsync);
      Ns *= R;
      nsh = (nsh >= 0 && (R & (R - 1)) == 0) ? nsh + (R == 8 ? 3 : R == 4 ? 2 : 1) : -1;
    }
  }
}

// padded index of element e in a row sequence (one spare slot per 8 elements)
__host__ __device__ __forceinline__ int rpad(int e) { return e + (e >> 3); }
__host__ __device__ __forceinline__ int rpitch(int n) { return n + (n >> 3) + 1; }

#define HS_FFT_ROWS(INV, buf, pitch, nseq, plan, tw, tid, nthr)                                       \
  ::hs::fft_smem<INV, false>(buf, pitch, 1, 3, nseq, (plan).L, (plan).nstage, (plan).packed, tw, tid, nthr)
// a plan with a radix-5, 7 or 11 stage
__host__ __device__ inline bool plan_ext(const FftPlan& p) {
  for (int st = 0; st < p.nstage; ++st) {
    const int R = (p.packed >> (4 * st)) & 15;
    if (R == 5 || R == 7 || R == 11) return true;
  }
  return false;
}

#define HS_FFT_COLS(INV, buf, W, nseq, plan, tw, tid, nthr) \
  ::hs::fft_smem<INV, true>(buf, 1, W, -1, nseq, (plan).L, (plan).nstage, (plan).packed, tw, tid, nthr)


// ---------------------------------------------------------------------------
// Compile-time plans for the hot lengths: every stride, stage count and
// radix is a constant, so the per-element index arithmetic folds away.
// ---------------------------------------------------------------------------
template <int L> struct FixedPlan { static constexpr int n = 0; };
template <> struct FixedPlan<64> {
  static constexpr int n = 2;
  __host__ __device__ static constexpr int r(int i) { return 8; }
};
template <> struct FixedPlan<128> {
  static constexpr int n = 3;
  __host__ __device__ static constexpr int r(int i) { return i == 0 ? 8 : 4; }
};
template <> struct FixedPlan<256> {
  static constexpr int n = 3;
  __host__ __device__ static constexpr int r(int i) { return i == 2 ? 4 : 8; }
};
template <> struct FixedPlan<512> {
  static constexpr int n = 3;
  __host__ __device__ static constexpr int r(int i) { return 8; }
};

// Position of element e inside a sequence: e*ES + (e >> PS) for PS >= 0, e*ES
// for PS = -1, and for PS = -2 (rows, ES = 1, length a multiple of 16) the XOR
// swizzle e ^ (((e >> 2) ^ (e >> 3)) & 15), a permutation of each row that keeps
// the 64-bit accesses of every stage of the fixed 64..512 plans within 3% of
// conflict-free (rows of length 64 are spaced 72 apart; see rowpass.cuh).
template <int ES, int PS> __host__ __device__ __forceinline__ int seq_pos(int e) {
  if constexpr (PS == -2) return e ^ (((e >> 2) ^ (e >> 3)) & 15);
  else return e * ES + (PS >= 0 ? (e >> PS) : 0);
}
__host__ __device__ __forceinline__ int rswz(int e) { return seq_pos<1, -2>(e); }

// The row swizzle is linear over XOR (shifts, XOR and masks are), and an index that is a sum of
// parts with disjoint bits is their XOR, so swz(a + b) = swz(a) ^ swz(b) for such parts: a
// thread swizzles its own offset once per stage and each element adds one XOR with a constant.
__host__ __device__ constexpr int swz_c(int e) { return e ^ (((e >> 2) ^ (e >> 3)) & 15); }
__host__ __device__ constexpr int ilog2_c(int v) { return v <= 1 ? 0 : 1 + ilog2_c(v >> 1); }
// b = pq NS + kk (kk < NS) -> pq NS R + kk: the bits of b at and above log2 NS move up by log2 R
template <int NS, int R> __device__ __forceinline__ int stockham_out(int b) {
  return ((b >> ilog2_c(NS)) << (ilog2_c(NS) + ilog2_c(R))) | (b & (NS - 1));
}

// Twiddle table of a fixed plan in shared memory, laid out per stage: stage s (NS_s = r_0 ... r_{s-1}
// > 1) needs w_L^{kk m step_s} for m = 1 .. R_s - 1 and kk < NS_s, kept at entry
// NS_s - r_0 + (m - 1) NS_s + kk.  The lanes of a warp hold consecutive kk, so they read consecutive
// entries (no bank conflicts); since (R_s - 1) NS_s = NS_{s+1} - NS_s the stages follow each other
// and the table has L - r_0 entries.
template <int L, typename C>
__device__ __forceinline__ void stage_twiddles(C* tab, const C* __restrict__ tw, int tid, int nthr) {
  constexpr int R0 = FixedPlan<L>::r(0);
  for (int j = tid; j < L - R0; j += nthr) {
    int ns = R0, st = 1;
    while (st + 1 < FixedPlan<L>::n && j >= ns * FixedPlan<L>::r(st) - R0) {
      ns *= FixedPlan<L>::r(st);
      ++st;
    }
    const int i = j - (ns - R0);
    const int m = i / ns + 1, kk = i - (m - 1) * ns;
    tab[j] = __ldg(tw + kk * m * (L / (ns * FixedPlan<L>::r(st))));
  }
}
// twiddle m of butterfly kk in the stage with NS and step: from the per-stage table in shared
// memory (TWS), or from the plain table through the read-only path
template <bool TWS, int L, int NS, typename C>
__device__ __forceinline__ C stage_tw(const C* __restrict__ tw, int m, int kk, int step) {
  if constexpr (TWS) return tw[(NS - FixedPlan<L>::r(0)) + (m - 1) * NS + kk];
  else return __ldg(tw + kk * m * step);
}

// twiddle i of the table: from global memory through the read-only path, or (TWS) from a copy
// of the table in shared memory
template <bool TWS, typename C> __device__ __forceinline__ C tw_load(const C* __restrict__ tw, int i) {
  if constexpr (TWS) {
    return tw[i];
  } else {
    return __ldg(tw + i);
  }
}

// one stage; sequence s element e at buf[s*SS + seq_pos<ES, PS>(e)]
template <int L, int R, int NS, int SS, int ES, int PS, bool INV, bool TWS = false, typename C>
__device__ __forceinline__ void stage_fixed(C* buf, int s, int t, bool active, const C* __restrict__ tw, bool wsync) {
  constexpr int T = L / kE;
  constexpr int nb = L / R;
  constexpr int KB = (nb + T - 1) / T;
  constexpr int step = L / (NS * R);
  // swizzled rows (PS = -2): T, nb, NS and R are powers of two and t < T, so the loads' index
  // b + m nb = t + k T + m nb and the stores' pq NS R + kk + m NS split into disjoint parts
  constexpr bool XS = (PS == -2) && (T & (T - 1)) == 0 && (nb & (nb - 1)) == 0 && (NS & (NS - 1)) == 0 &&
                      (R & (R - 1)) == 0;
  const int tin = XS ? swz_c(t) : 0;
  const int tout = XS ? swz_c(stockham_out<NS, R>(t)) : 0;
  C v[KB][R];
  C* sb = buf + s * SS;
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int b = t + k * T;
    if (active && b < nb) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int e = b + m * nb;
        if constexpr (XS) v[k][m] = sb[tin ^ swz_c(k * T + m * nb)];
        else v[k][m] = sb[seq_pos<ES, PS>(e)];
      }
    }
  }
  if (wsync) __syncwarp(); else __syncthreads();
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int b = t + k * T;
    if (active && b < nb) {
      const int kk = b & (NS - 1);
      const int pq = b / NS;
      if (NS > 1) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          C w = stage_tw<TWS, L, NS>(tw, m, kk, step);
          if (INV) w.y = -w.y;
          v[k][m] = cmul(v[k][m], w);
        }
      }
      Dft<R, INV, C>::run(v[k]);
      const int base = pq * NS * R + kk;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int e = base + m * NS;
        if constexpr (XS) sb[tout ^ swz_c(stockham_out<NS, R>(k * T) + m * NS)] = v[k][m];
        else sb[seq_pos<ES, PS>(e)] = v[k][m];
      }
    }
  }
  if (wsync) __syncwarp(); else __syncthreads();
}

template <int L, int ST, int NS, int SS, int ES, int PS, bool INV, bool TWS = false, typename C>
__device__ __forceinline__ void stages_fixed(C* buf, int s, int t, bool active, const C* __restrict__ tw,
                                             bool wsync) {
  if constexpr (ST < FixedPlan<L>::n) {
    constexpr int R = FixedPlan<L>::r(ST);
    stage_fixed<L, R, NS, SS, ES, PS, INV, TWS>(buf, s, t, active, tw, wsync);
    stages_fixed<L, ST + 1, NS * R, SS, ES, PS, INV, TWS>(buf, s, t, active, tw, wsync);
  }
}

// Same contract as fft_smem with L, the strides and the mapping fixed at compile time.  TWS: tw
// points to the plan's per-stage twiddle table in shared memory (stage_twiddles).
template <int L, bool INV, bool COLMAP, int SS, int ES, int PS, bool TWS = false, typename C>
__device__ __forceinline__ void fft_fixed(C* buf, int nseq, const C* __restrict__ tw, int tid, int nthreads) {
  constexpr int T = L / kE;
  const int G = nthreads / T;
  const bool wsync = !COLMAP && T <= 32 && (32 % T) == 0 && (nthreads % 32) == 0;
  for (int g0 = 0; g0 < nseq; g0 += G) {
    const int sl = COLMAP ? (tid % G) : (tid / T);
    const int t = COLMAP ? (tid / G) : (tid % T);
    const int s = g0 + sl;
    const bool active = (COLMAP ? (t < T) : (sl < G)) && s < nseq;
    stages_fixed<L, 0, 1, SS, ES, PS, INV, TWS>(buf, s, t, active, tw, wsync);
  }
}


// ---------------------------------------------------------------------------
// Column-tile FFTs with global-memory ends: sequence s = c * CT + col (c the
// field component, col the column in the tile) is column col of component c,
// element e of it lives at g[c * cstride + col + e * rstride] in global memory
// and at sm[e * W + s] in the shared tile.  IN_G: the first stage reads its
// butterfly inputs from global memory (columns >= ccols read as zero); OUT_G:
// the last stage writes its outputs to global memory (columns < ncol only).
// Every other stage goes through the shared tile as in fft_fixed (COLMAP).
// ---------------------------------------------------------------------------
template <typename C> struct ColIO {
  const C* gin;
  C* gout;
  size_t cstride, rstride;
  int ccols, ncol;
};

template <int L, int R, int NS, int W, int CT, bool INV, bool FROM_G, bool TO_G, bool TWS = false, typename C>
__device__ __forceinline__ void stage_col(C* sm, const ColIO<C>& io, int s, int t, bool active,
                                          const C* __restrict__ tw) {
  constexpr int T = L / kE;
  constexpr int nb = L / R;
  constexpr int KB = (nb + T - 1) / T;
  constexpr int step = L / (NS * R);
  const int c = s / CT, col = s - c * CT;
  C v[KB][R];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int b = t + k * T;
    if (active && b < nb) {
      if (FROM_G) {
        const C* gp = io.gin + c * io.cstride + col;
        const bool ok = col < io.ccols;
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const int e = b + m * nb;
          v[k][m] = ok ? gp[(size_t)e * io.rstride] : cmk<C>(0, 0);
        }
      } else {
#pragma unroll
        for (int m = 0; m < R; ++m) v[k][m] = sm[(b + m * nb) * W + s];
      }
    }
  }
  if (!FROM_G) __syncthreads();
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int b = t + k * T;
    if (active && b < nb) {
      const int kk = b & (NS - 1);
      const int pq = b / NS;
      if (NS > 1) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          C w = stage_tw<TWS, L, NS>(tw, m, kk, step);
          if (INV) w.y = -w.y;
          v[k][m] = cmul(v[k][m], w);
        }
      }
      Dft<R, INV, C>::run(v[k]);
      const int base = pq * NS * R + kk;
      if (TO_G) {
        if (col < io.ncol) {
          C* gp = io.gout + c * io.cstride + col;
#pragma unroll
          for (int m = 0; m < R; ++m) gp[(size_t)(base + m * NS) * io.rstride] = v[k][m];
        }
      } else {
#pragma unroll
        for (int m = 0; m < R; ++m) sm[(base + m * NS) * W + s] = v[k][m];
      }
    }
  }
  if (!TO_G) __syncthreads();
}

template <int L, int ST, int NS, int W, int CT, bool INV, bool IN_G, bool OUT_G, bool TWS = false, typename C>
__device__ __forceinline__ void stages_col(C* sm, const ColIO<C>& io, int s, int t, bool active,
                                           const C* __restrict__ tw) {
  if constexpr (ST < FixedPlan<L>::n) {
    constexpr int R = FixedPlan<L>::r(ST);
    constexpr bool FIRST = (ST == 0), LAST = (ST + 1 == FixedPlan<L>::n);
    stage_col<L, R, NS, W, CT, INV, IN_G && FIRST, OUT_G && LAST, TWS>(sm, io, s, t, active, tw);
    stages_col<L, ST + 1, NS * R, W, CT, INV, IN_G, OUT_G, TWS>(sm, io, s, t, active, tw);
  }
}

// FFT of the W = 3 * CT columns of a tile; lanes walk across columns (COLMAP).
// TWS: tw points to the plan's per-stage twiddle table in shared memory (stage_twiddles).
template <int L, int W, int CT, bool INV, bool IN_G, bool OUT_G, bool TWS = false, typename C>
__device__ __forceinline__ void fft_col_fixed(C* sm, const ColIO<C>& io, const C* __restrict__ tw, int tid,
                                              int nthreads) {
  constexpr int T = L / kE;
  const int G = nthreads / T;
  for (int g0 = 0; g0 < W; g0 += G) {
    const int sl = tid % G, t = tid / G;
    const int s = g0 + sl;
    const bool active = t < T && s < W;
    stages_col<L, 0, 1, W, CT, INV, IN_G, OUT_G, TWS>(sm, io, s, t, active, tw);
  }
}

}  // namespace hs
