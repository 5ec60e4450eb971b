// hs_residual_noalloc: the FP64 equilibrium residual of a displacement field,
// computed without any device allocation.
//
// Who needs this: code that may not allocate device memory at the moment it
// runs - real-time or embedded callers that run inside a fixed, pre-reserved
// memory budget, callers whose device memory is wholly owned by another
// allocator (a framework's caching pool, where a stray cudaMalloc would
// fragment or exceed what that pool manages), and checks run from places where
// an allocation could fail or stall (inside an out-of-memory handler, a
// watchdog).  Such callers cannot provide the workspace that hs_create needs, so
// this entry point keeps the little scratch it uses (the device copy of the
// phase table, per-block partial sums and a status record) in one file-scope
// device array of fixed size that exists for as long as the library is
// loaded.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/hs.h"
#include "launch.h"

namespace {

// Layout of the scratch array: status record | phase table | block partials.
constexpr size_t kStatusBytes = 256;
constexpr size_t kTableBytes = (size_t)HS_NOALLOC_MAX_PHASES * 21 * sizeof(double);
constexpr size_t kPartialBytes = (size_t)HS_NOALLOC_MAX_BLOCKS * hs::NRED * sizeof(double);
constexpr size_t kScratchBytes = kStatusBytes + kTableBytes + kPartialBytes;
static_assert(kScratchBytes <= HS_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");
// The last int of the status block receives the largest phase id of the call.
constexpr size_t kMaxIdOffset = kStatusBytes - sizeof(int);
static_assert(sizeof(hs::DevStatus) + sizeof(double) <= kMaxIdOffset, "status record too large");

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices];  // device address of g_noalloc_scratch per device ordinal

// The device-side address of the array, looked up once per device with that
// device current.  (In host code the array's name is only a host stand-in.)
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

bool isotropic(const double* C, double* lam, double* mu) {
  double scale = 0;
  for (int i = 0; i < 36; ++i) scale = std::max(scale, std::fabs(C[i]));
  const double tol = 1e-12 * std::max(scale, 1e-300);
  const double l = C[1], m = C[21];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double want = 0;
      if (i < 3 && j < 3) want = (i == j) ? l + 2 * m : l;
      else if (i == j) want = m;
      if (std::fabs(C[i * 6 + j] - want) > tol) return false;
    }
  *lam = l;
  *mu = m;
  return true;
}

// The grids hs_create accepts: even, 4..512, prime factors 2, 3, 5, 7 and 11 (the
// real-space pass itself needs no FFT plan, so every such length runs).
bool supported(int n) {
  if (n < 4 || n > 512 || (n % 2) != 0) return false;
  for (int f : {2, 3, 5, 7, 11})
    while (n % f == 0) n /= f;
  return n == 1;
}

}  // namespace

extern "C" hs_status hs_residual_noalloc(const int grid[3], const unsigned short* ids, const double* table,
                                         int nphase, const double E[6], const double* u, float* force,
                                         double sig_mean[6], double* l2, void* stream) {
  if (!grid || !ids || !table || !E || !u || !sig_mean || !l2) return HS_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    if (!supported(grid[i])) return HS_ERR_UNSUPPORTED_SIZE;
  if (nphase < 1 || nphase > HS_NOALLOC_MAX_PHASES) return HS_ERR_INVALID_ARG;
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(E[i])) return HS_ERR_INVALID_ARG;
  const int n1 = grid[0], n2 = grid[1], n3 = grid[2];
  const int nthr = ((n1 + 31) / 32) * 32;
  // rows per block: 4 where N2 allows, halved while the plane ring does not fit
  // in the device's opt-in shared memory (N1 = 512 needs 2)
  int dev = 0, smem_optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return HS_ERR_CUDA;
  int ty = (n2 % 4 == 0) ? 4 : 2;
  size_t smem = hs::march_layout(n1, 0, nthr, ty, hs::MODE_FORCE, true, false, 8).total;
  while (ty > 2 && smem > (size_t)smem_optin) {
    ty /= 2;
    smem = hs::march_layout(n1, 0, nthr, ty, hs::MODE_FORCE, true, false, 8).total;
  }
  if (smem > (size_t)smem_optin) return HS_ERR_UNSUPPORTED_SIZE;
  const int ytiles = n2 / ty;
  int nzc = std::max(1, std::min(n3, (608 + ytiles - 1) / ytiles));
  const int zc = (n3 + nzc - 1) / nzc;
  nzc = (n3 + zc - 1) / zc;
  if ((size_t)ytiles * nzc > (size_t)HS_NOALLOC_MAX_BLOCKS) return HS_ERR_UNSUPPORTED_SIZE;

  // phase table in the kernel's layout
  bool iso = true;
  static thread_local double packed[(size_t)HS_NOALLOC_MAX_PHASES * 21];
  for (int p = 0; p < nphase; ++p) {
    double lam, mu;
    if (!isotropic(table + (size_t)p * 36, &lam, &mu)) iso = false;
  }
  for (int p = 0; p < nphase; ++p) {
    const double* C = table + (size_t)p * 36;
    for (int i = 0; i < 36; ++i)
      if (!std::isfinite(C[i])) return HS_ERR_INVALID_ARG;
    if (iso) {
      double lam, mu;
      isotropic(C, &lam, &mu);
      packed[2 * p] = lam;
      packed[2 * p + 1] = mu;
    } else {
      int k = 0;
      for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) packed[(size_t)p * 21 + k++] = C[i * 6 + j];
    }
  }

  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return HS_ERR_CUDA;
  hs::DevStatus* st = reinterpret_cast<hs::DevStatus*>(base);
  double* hist = reinterpret_cast<double*>(base + sizeof(hs::DevStatus));
  double* mat = reinterpret_cast<double*>(base + kStatusBytes);
  double* partials = reinterpret_cast<double*>(base + kStatusBytes + kTableBytes);

  int* maxid = reinterpret_cast<int*>(base + kMaxIdOffset);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nvox = (size_t)n1 * n2 * n3;

  // The array keeps the previous call's contents: reset the status record
  // (block-arrival counter, flags) and the max-id slot, and load this call's
  // phase table.
  unsigned char head[kStatusBytes];
  memset(head, 0, sizeof(head));
  hs::DevStatus h;
  memset(&h, 0, sizeof(h));
  h.max_iter = 1 << 30;
  h.hist_cap = 1;
  h.nvox = (double)nvox;
  memcpy(head, &h, sizeof(h));
  e = cudaMemcpyAsync(base, head, kStatusBytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mat, packed, (size_t)nphase * (iso ? 2 : 21) * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return HS_ERR_CUDA;
  // Every id must index the table: the stress kernel reads the table at the
  // id without a bound, so an id >= nphase is refused before it runs.
  int hmax = 0;
  e = hs::launch_max_id(ids, nvox, maxid, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hmax, maxid, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return HS_ERR_CUDA;
  if (hmax >= nphase) return HS_ERR_INVALID_ARG;

  hs::MarchArgs<double> a;
  memset(&a, 0, sizeof(a));
  a.ids = ids;
  a.mat = mat;
  for (int i = 0; i < 6; ++i) a.E[i] = E[i];
  a.n1 = n1;
  a.n2 = n2;
  a.n3 = n3;
  a.P = n1 / 2 + 1;
  a.zc = zc;
  a.partials = partials;
  a.st = st;
  a.hist = hist;
  a.ureal = u;
  a.fout = force;
  a.fout_f32 = 1;
  a.skip_if_done = 0;
  e = hs::launch_march<double>(a, iso, ty, hs::MODE_FORCE, true, dim3(ytiles, nzc), nthr, smem, s);
  if (e != cudaSuccess) return HS_ERR_CUDA;
  e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return HS_ERR_CUDA;
  for (int i = 0; i < 6; ++i) sig_mean[i] = h.sig_mean[i];
  *l2 = h.l2;
  return HS_OK;
}
