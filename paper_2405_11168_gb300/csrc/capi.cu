// Host side of the C ABI declared in include/hs.h.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <unordered_map>
#include <functional>
#include <vector>

#include <cuda.h>  // tensor-map types; the encoder is fetched through the runtime
#include <cudaTypedefs.h>

#include "../../include/hs.h"
#include "launch.h"

using hs::DevStatus;
using hs::FftPlan;

namespace {

thread_local std::string g_last_error;

constexpr int kHistCap = 1 << 16;
constexpr int kMaxN = 512;
// Real-space pass blocks: ~7 per SM (z chunks of 16 planes at 256^3).  Longer
// chunks re-read fewer halo planes; measured on GB300 at 256^3 (TY = 4):
// 0.327 / 0.283 / 0.266 / 0.261 / 0.270 / 0.280 ms for chunks of 4 / 8 / 12 / 16 / 24 / 32.
constexpr int kTargetBlocks = 1024;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool make_plan(int L, FftPlan* p) {
  p->L = L;
  p->nstage = 0;
  p->packed = 0;
  int r = L;
  auto push = [&](int R) {
    if (p->nstage >= hs::kMaxStages) return false;
    p->packed |= R << (4 * p->nstage);
    p->nstage++;
    r /= R;
    return true;
  };
  while (r % 8 == 0)
    if (!push(8)) return false;
  while (r % 4 == 0)
    if (!push(4)) return false;
  while (r % 2 == 0)
    if (!push(2)) return false;
  while (r % 3 == 0)
    if (!push(3)) return false;
  for (int R : {5, 7, 11})
    while (r % R == 0)
      if (!push(R)) return false;
  return r == 1 && p->nstage > 0;
}

// w_L^j = exp(-2 pi i j / L), j < L, with exact values on the quarter points
void twiddles(int L, std::vector<double>& re, std::vector<double>& im) {
  re.resize(L);
  im.resize(L);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int j = 0; j < L; ++j) {
    if ((4 * j) % L == 0) {
      const int q = (4 * j) / L;  // quarter turns
      static const double cr[4] = {1, 0, -1, 0}, ci[4] = {0, -1, 0, 1};
      re[j] = cr[q];
      im[j] = ci[q];
      continue;
    }
    const long double t = 2.0L * pi * (long double)j / (long double)L;
    re[j] = (double)cosl(t);
    im[j] = (double)-sinl(t);
  }
}

// Voigt index of tensor pair (i, j), order 11,22,33,23,13,12
int vidx(int i, int j) {
  static const int V[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
  return V[i][j];
}

bool is_isotropic(const double* C, double* lam, double* mu) {
  double scale = 0;
  for (int i = 0; i < 36; ++i) scale = std::max(scale, fabs(C[i]));
  const double tol = 1e-12 * std::max(scale, 1e-300);
  const double l = C[1], m = C[21];  // C[0][1], C[3][3]
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double want = 0;
      if (i < 3 && j < 3) want = (i == j) ? l + 2 * m : l;
      else if (i == j) want = m;
      if (fabs(C[i * 6 + j] - want) > tol) return false;
    }
  *lam = l;
  *mu = m;
  return true;
}

// eigenvalues of a symmetric n x n matrix (cyclic Jacobi), n <= 6
void sym_eig(std::vector<double> a, int n, std::vector<double>& ev) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (fabs(apq) < 1e-300) continue;
        const double theta = (a[q * n + q] - a[p * n + p]) / (2 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
        const double c = 1 / sqrt(t * t + 1), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
}

// Voigt bulk modulus and the range of deviatoric eigenvalues (Mandel form)
void bulk_and_shear_range(const double* C, double* K, double* dmin, double* dmax) {
  double s = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) s += C[i * 6 + j];
  *K = s / 9.0;
  const double r2 = sqrt(2.0);
  double M[36];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) M[i * 6 + j] = C[i * 6 + j] * (i < 3 ? 1 : r2) * (j < 3 ? 1 : r2);
  // orthonormal basis of the deviatoric subspace
  double B[5][6] = {{1 / r2, -1 / r2, 0, 0, 0, 0},
                    {1 / sqrt(6.0), 1 / sqrt(6.0), -2 / sqrt(6.0), 0, 0, 0},
                    {0, 0, 0, 1, 0, 0},
                    {0, 0, 0, 0, 1, 0},
                    {0, 0, 0, 0, 0, 1}};
  std::vector<double> D(25, 0.0);
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      double v = 0;
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) v += B[a][i] * M[i * 6 + j] * B[b][j];
      D[a * 5 + b] = v;
    }
  std::vector<double> ev;
  sym_eig(D, 5, ev);
  *dmin = *std::min_element(ev.begin(), ev.end());
  *dmax = *std::max_element(ev.begin(), ev.end());
}

void iso_voigt(double lam, double mu, double* C) {
  for (int i = 0; i < 36; ++i) C[i] = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i * 6 + j] = (i == j) ? lam + 2 * mu : lam;
  for (int i = 3; i < 6; ++i) C[i * 6 + i] = mu;
}

bool cholesky_pd(const double* A) {
  double L[36] = {0};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[i * 6 + j];
      for (int k = 0; k < j; ++k) s -= L[i * 6 + k] * L[j * 6 + k];
      if (i == j) {
        if (!(s > 0)) return false;
        L[i * 6 + i] = sqrt(s);
      } else {
        L[i * 6 + j] = s / L[j * 6 + j];
      }
    }
  return true;
}

struct Layout {
  size_t S, B0, B1, F, ids, matk, matd, tw, partials, status, hist, macro, sig0f, sig0d, c0, u64, rsrc, total;
};

}  // namespace

struct hs_ctx {
  int n1, n2, n3, nh, P;
  size_t N;
  int prec;
  bool f64;  // iteration kernels in FP64
  hs_options opt;
  cudaStream_t stream;
  int nphase;
  bool iso;
  std::vector<double> table;
  double C0[36];
  double G6[36];
  bool c0_iso = false;      // the reference medium is isotropic: Omega^-1 = c0_a M + c0_b tr(M) I
  double c0_a = 0, c0_b = 0;
  // batched launches (hs_batch): the kernels of this context run over batch_n items whose
  // workspaces follow one another batch_stride bytes apart (1 and 0 for a single solve)
  int batch_n = 1;
  size_t batch_stride = 0;
  int layout_np = 1;        // phase count the workspace layout was sized for (>= nphase)
  bool unbound = false;     // a failed hs_set_material left the workspace without a valid material
  char* ws;
  size_t ws_bytes;
  Layout lay;
  void* S;
  void* B[2];  // xfuse: ping-pong spectral buffers; split: B[0] spectral work, B[1] real displacement
  void* F;     // split: real force
  uint16_t* ids;
  void* matk;
  double* matd;
  void* twk[3];
  double* partials;
  DevStatus* st;
  double* hist;
  double* u64;
  float* rsrc;
  double* macro;   // device [sigma^a (6), S0 (36)] of the applied-stress loop
  float* sig0f;    // device lambda(p) : eps0(p), Voigt, per phase (eigenstrain)
  double* sig0d;
  bool has_eigen = false;
  // captured iteration chunks: [0] full problem, [1] correction solves (refined)
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int gchunks[2] = {0, 0};   // uncaptured chunks run so far (capture follows the first)
  long long glaunches[2][HS_K_COUNT] = {};  // kernel launches per replay, by class
  bool capturing = false;                    // inside the stream capture of chunk cap_gi
  int cap_gi = 0;
  bool dev_macro = false;    // plain modes under applied stress: E lives in the device status
  double Einit[6] = {0, 0, 0, 0, 0, 0};
  FftPlan plan[3];
  int ty, zc, nthr_m;
  dim3 grid_m;
  int ty64;       // y rows per block of the FP64 residual sweep (refined mode)
  int zc64;
  dim3 grid_m64;
  int ct, nthr_y, nthr_z;
  bool xfuse;
  int nthr_row, nblk_row[2];  // [ROW_C2R], [ROW_R2C]
  size_t smem_row[2];
  size_t smem_y, smem_z;
  bool zstate_smem = false;  // the z pass copies the state tile to shared memory
  // persistent double-buffered y / z passes (k_colp): blocks and shared memory
  bool pipe_y = false, pipe_z = false;
  // column passes fed by tensor copies: the tile map of work buffer B[b] for the y (axis 0)
  // and z (axis 1) passes, cached with the base, item stride and item count it was made for
  CUtensorMap tmap[2][2];
  const void* tmap_base[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  size_t tmap_stride[2][2] = {{0, 0}, {0, 0}};
  int tmap_n[2][2] = {{0, 0}, {0, 0}};
  bool tmap_ok[2][2] = {{false, false}, {false, false}};
  int nblk_py = 0, nblk_pz = 0;
  size_t smem_py = 0, smem_pz = 0;
  dim3 grid_y, grid_z;
  bool warm;
  int cur;
  std::vector<double> hist_host;
  std::string last_err;
  // profiling
  bool prof;
  long long launches[HS_K_COUNT];
  struct Ev { int kind; cudaEvent_t a, b; };
  std::vector<Ev> ev_used;
  std::vector<cudaEvent_t> ev_pool;
  int prof_every = 1;                // kernel events in one iteration chunk of every prof_every
  bool prof_skip = false;            // this chunk records no kernel events
  long long chunk_seq = 0;           // iteration chunks run with profiling on
  long long timed[HS_K_COUNT] = {};  // launches that recorded events, by class
};

namespace {

hs_status fail(hs_ctx* c, hs_status s, const std::string& msg) {
  g_last_error = msg;
  if (c) c->last_err = msg;
  return s;
}

hs_status cuda_fail(hs_ctx* c, cudaError_t e, const char* where) {
  return fail(c, HS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// A launch grid extended over the items of a batched context.
dim3 zg(const hs_ctx* c, dim3 g) {
  g.z = (unsigned)c->batch_n;
  return g;
}

// Bracket one kernel launch: count it and, when profiling, record events.  Inside
// the stream capture of an iteration chunk the launch is counted once per replay
// instead, and records no events (a profiled chunk runs as plain launches).
struct LaunchScope {
  hs_ctx* c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  LaunchScope(hs_ctx* c_, int kind_) : c(c_), kind(kind_) {
    if (c->capturing) c->glaunches[c->cap_gi][kind]++;
    else c->launches[kind]++;
    if (c->prof && !c->capturing && !c->prof_skip) {
      a = take();
      b = take();
      if (a) cudaEventRecord(a, c->stream);
    }
  }
  cudaEvent_t take() {
    cudaEvent_t e = nullptr;
    if (!c->ev_pool.empty()) {
      e = c->ev_pool.back();
      c->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
    }
    return e;
  }
  ~LaunchScope() {
    if (a && b) {
      cudaEventRecord(b, c->stream);
      c->ev_used.push_back({kind, a, b});
      c->timed[kind]++;
    } else {
      if (a) c->ev_pool.push_back(a);
      if (b) c->ev_pool.push_back(b);
    }
  }
};

// Forget captured chunk gi: its graph and its launch counts.
void drop_graph(hs_ctx* c, int gi, bool reset_chunks) {
  if (c->gexec[gi]) cudaGraphExecDestroy(c->gexec[gi]);
  c->gexec[gi] = nullptr;
  for (int k = 0; k < HS_K_COUNT; ++k) c->glaunches[gi][k] = 0;
  if (reset_chunks) c->gchunks[gi] = 0;
}

// A replay of chunk gi was enqueued: count its kernel launches.
void account_replay(hs_ctx* c, int gi) {
  for (int k = 0; k < HS_K_COUNT; ++k) c->launches[k] += c->glaunches[gi][k];
}

// Clears the per-chunk profiling switch on every exit from the iteration loop.
struct ChunkProfGuard {
  hs_ctx* c;
  ~ChunkProfGuard() { c->prof_skip = false; }
};

#define HS_CU(c, call)                                    \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return cuda_fail(c, _e, #call); \
  } while (0)

// Exact compression of a per-voxel stiffness field into phase ids and a phase
// table: voxels whose 21 coefficients are bit-identical (-0 read as +0) share a
// phase, numbered in order of first appearance.  Voxels are fed in memory order
// (x fastest), a run of planes at a time.
class CoeffCompressor {
 public:
  CoeffCompressor(size_t nvox, int capacity) : ids(nvox), cap_(capacity) {}
  // comp[c] points at coefficient c of `count` consecutive voxels starting at voxel `base`
  hs_status add(const float* const comp[21], size_t count, size_t base) {
    for (size_t v = 0; v < count; ++v) {
      Key k;
      for (int c = 0; c < 21; ++c) {
        float f = comp[c][v];
        if (!std::isfinite(f)) return HS_ERR_INVALID_ARG;
        if (f == 0.0f) f = 0.0f;  // -0 and +0 are the same stiffness
        memcpy(&k.w[c], &f, 4);
      }
      int id;
      if (prev_id_ >= 0 && k == prev_) {
        id = prev_id_;  // fast path: grains are runs along x
      } else {
        auto it = index_.find(k);
        if (it != index_.end()) {
          id = it->second;
        } else {
          if ((int)index_.size() >= cap_) return HS_ERR_UNSUPPORTED_SIZE;
          id = (int)index_.size();
          index_.emplace(k, id);
          table.resize(table.size() + 36);
          double* C = &table[(size_t)id * 36];
          int t = 0;
          for (int i = 0; i < 6; ++i)
            for (int j = i; j < 6; ++j) {
              float f;
              memcpy(&f, &k.w[t++], 4);
              C[i * 6 + j] = C[j * 6 + i] = (double)f;
            }
        }
      }
      ids[base + v] = (uint16_t)id;
      prev_ = k;
      prev_id_ = id;
    }
    return HS_OK;
  }
  int nphase() const { return (int)index_.size(); }
  std::vector<uint16_t> ids;
  std::vector<double> table;

 private:
  struct Key {
    uint32_t w[21];
    bool operator==(const Key& o) const { return memcmp(w, o.w, sizeof(w)) == 0; }
  };
  struct KeyHash {
    size_t operator()(const Key& k) const {
      uint64_t h = 1469598103934665603ull;  // FNV-1a over the coefficient bits
      for (int i = 0; i < 21; ++i) {
        h ^= k.w[i];
        h *= 1099511628211ull;
      }
      return (size_t)h;
    }
  };
  std::unordered_map<Key, int, KeyHash> index_;
  Key prev_{};
  int prev_id_ = -1;
  int cap_;
};

// A material in ids form: kind HS_COEFFS_F32 is compressed (its coefficients read
// from host or device memory a z plane at a time); other kinds pass through.
struct IdsMaterial {
  std::vector<uint16_t> ids;
  std::vector<double> table;
  hs_material m{};
  const hs_material* use = nullptr;
};

hs_status to_ids_material(const hs_material* in, const int grid[3], void* stream, IdsMaterial* out) {
  if (in->kind != HS_COEFFS_F32) {
    out->use = in;
    return HS_OK;
  }
  if (!in->coeffs) return HS_ERR_INVALID_ARG;
  const size_t plane = (size_t)grid[0] * grid[1], N = plane * grid[2];
  CoeffCompressor cc(N, HS_MAX_PHASES);
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, in->coeffs);
  const bool dev_ptr = (e == cudaSuccess) && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
  if (e != cudaSuccess) cudaGetLastError();
  const float* comp[21];
  if (!dev_ptr) {
    for (int c = 0; c < 21; ++c) comp[c] = in->coeffs + (size_t)c * N;
    hs_status s = cc.add(comp, N, 0);
    if (s != HS_OK) return s;
  } else {
    std::vector<float> buf(21 * plane);
    for (int c = 0; c < 21; ++c) comp[c] = buf.data() + (size_t)c * plane;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int z = 0; z < grid[2]; ++z) {
      // the 21 coefficient planes of z: one strided copy
      e = cudaMemcpy2DAsync(buf.data(), plane * 4, in->coeffs + (size_t)z * plane, N * 4, plane * 4, 21,
                            cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        g_last_error = std::string("coefficient read: ") + cudaGetErrorString(e);
        return HS_ERR_CUDA;
      }
      hs_status s = cc.add(comp, plane, (size_t)z * plane);
      if (s != HS_OK) return s;
    }
  }
  out->ids = std::move(cc.ids);
  out->table = std::move(cc.table);
  out->m.kind = HS_IDS_U16;
  out->m.ids = out->ids.data();
  out->m.table = out->table.data();
  out->m.nphase = cc.nphase();
  out->m.coeffs = nullptr;
  out->use = &out->m;
  return HS_OK;
}

hs_status check_grid(const int grid[3]) {
  for (int i = 0; i < 3; ++i) {
    const int n = grid[i];
    if (n < 4 || n > kMaxN || (n % 2) != 0) return HS_ERR_UNSUPPORTED_SIZE;
    FftPlan p;
    if (!make_plan(n, &p)) return HS_ERR_UNSUPPORTED_SIZE;
  }
  return HS_OK;
}

int pitch_of(int nh, bool f64) { return f64 ? ((nh + 1) & ~1) : ((nh + 3) & ~3); }

int pick_ty(int n2) { return (n2 % 4 == 0) ? 4 : 2; }

// z chunk of an FP64 real-space pass.  Its blocks (one per (y tile, z chunk), launched y tile
// first) are bound by the FP64 pipe, so a block's time is proportional to the voxel layers it
// computes (chunk + 1) and the pass ends when a greedy list schedule of the blocks, in launch
// order, on the resident slots ends.  The chunk length with the earliest end is taken (the longer
// on ties: fewer recomputed layers).  At 256^3 on GB300 this model reproduces the measured
// sweep times of chunks 8..32 to 1%.
int pick_zchunk64(int yt, int n3, int slots) {
  int best_zc = 0;
  long long best = -1;
  std::vector<long long> heap(std::max(slots, 1));
  for (int zc = std::min(4, n3); zc <= std::min(n3, 64); ++zc) {
    std::fill(heap.begin(), heap.end(), 0LL);
    long long end = 0;
    const int nz = (n3 + zc - 1) / zc;
    for (int z = 0; z < nz; ++z) {
      const long long layers = std::min(zc, n3 - z * zc) + 1;
      for (int y = 0; y < yt; ++y) {
        std::pop_heap(heap.begin(), heap.end(), std::greater<long long>());
        heap.back() += layers;
        end = std::max(end, heap.back());
        std::push_heap(heap.begin(), heap.end(), std::greater<long long>());
      }
    }
    if (best < 0 || end < best || (end == best && zc > best_zc)) {
      best = end;
      best_zc = zc;
    }
  }
  return best_zc;
}

size_t march_smem(int n1, int ty, bool f64, int mode, bool real, bool has_src = false) {
  const int nh = n1 / 2 + 1;
  const int P = real ? 0 : pitch_of(nh, f64);
  const int nthr = ((n1 + 31) / 32) * 32;
  return hs::march_layout(n1, P, nthr, ty, mode, real, has_src, f64 ? 8 : 4).total;
}

Layout make_layout(int n1, int n2, int n3, int nphase, int prec) {
  Layout L;
  const bool f64 = (prec == HS_FP64);
  const int nh = n1 / 2 + 1, P = pitch_of(nh, f64);
  const size_t cs = f64 ? 16 : 8;
  const size_t N = (size_t)n1 * n2 * n3;
  const size_t cbuf = align256(std::max((size_t)3 * n3 * n2 * P * cs, 3 * N * (f64 ? 8 : 4)));
  const size_t max_blocks = (size_t)(n2 / 2) * n3;  // upper bound over y tiles and z-chunkings
  size_t off = 0;
  L.S = off; off += cbuf;
  L.B0 = off; off += cbuf;
  L.B1 = off; off += cbuf;
  L.F = off; off += cbuf;
  L.ids = off; off += align256(N * 2);
  L.matk = off; off += align256((size_t)nphase * 21 * (f64 ? 8 : 4));
  L.matd = off; off += align256((size_t)nphase * 21 * 8);
  L.tw = off; off += align256((size_t)(n1 + n2 + n3) * cs);
  L.partials = off; off += align256(max_blocks * hs::NRED * 8);
  L.status = off; off += align256(sizeof(DevStatus));
  L.hist = off; off += align256((size_t)kHistCap * 8);
  L.macro = off; off += align256(42 * 8);
  L.sig0f = off; off += align256((size_t)nphase * 6 * 4);
  L.sig0d = off; off += align256((size_t)nphase * 6 * 8);
  L.c0 = off; off += align256(32);  // isotropic reference medium (lambda0 + mu0, mu0): 2 double, then 2 float
  L.u64 = off;
  L.rsrc = off;
  if (prec == HS_FP32_REFINED) {
    L.u64 = off; off += align256(3 * N * 8);
    L.rsrc = off; off += align256(3 * N * 4);
  }
  L.total = off;
  return L;
}

template <typename T> void fill_march_common(hs_ctx* c, hs::MarchArgs<T>& a) {
  memset(&a, 0, sizeof(a));
  // full problem: eigenstrain and (plain modes) the device copy of E; the
  // refined path's correction solves clear both
  a.Edev = &c->st->E[0];
  a.sig0 = c->has_eigen ? (sizeof(T) == 8 ? (const T*)(const void*)c->sig0d : (const T*)(const void*)c->sig0f) : nullptr;
  a.ids = c->ids;
  a.mat = (const T*)(sizeof(T) == 8 && !c->f64 ? (void*)c->matd : c->matk);
  a.tw1 = (const typename hs::cplx_t<T>::type*)c->twk[0];
  a.plan1 = c->plan[0];
  a.n1 = c->n1;
  a.n2 = c->n2;
  a.n3 = c->n3;
  a.P = c->P;
  a.zc = c->zc;
  a.partials = c->partials;
  a.st = c->st;
  a.hist = c->hist;
  a.zstride = c->batch_stride;
}

template <typename T> void fill_col(hs_ctx* c, hs::ColArgs<T>& a, void* buf, int axis) {
  using C = typename hs::cplx_t<T>::type;
  memset(&a, 0, sizeof(a));
  a.buf = (C*)buf;
  a.S = (C*)c->S;
  a.tw = (const C*)c->twk[axis];
  a.tw1 = (const C*)c->twk[0];
  a.tw2 = (const C*)c->twk[1];
  a.tw3 = (const C*)c->twk[2];
  a.plan = c->plan[axis];
  a.n1 = c->n1;
  a.n2 = c->n2;
  a.n3 = c->n3;
  a.P = c->P;
  a.nh = c->nh;
  a.scale = (T)(2.0 / (double)c->N);
  for (int i = 0; i < 36; ++i) a.G6[i] = (T)c->G6[i];
  a.c0iso = c->c0_iso ? 1 : 0;
  a.c0a = (T)c->c0_a;
  a.c0b = (T)c->c0_b;
  // an isotropic reference medium is read from the workspace (per item in batched launches),
  // so captured iteration graphs stay valid when hs_set_material changes it
  if (c->c0_iso) a.c0dev = (const T*)(c->ws + c->lay.c0 + (sizeof(T) == 8 ? 0 : 16));
  a.st = c->st;
  a.skip_if_done = 1;
  a.zstride = c->batch_stride;
  a.state_smem = (axis == 2 && c->zstate_smem) ? 1 : 0;
}

template <typename T> hs_status launch_force(hs_ctx* c, const double E[6], int in, const float* src) {
  hs::MarchArgs<T> a;
  fill_march_common<T>(c, a);
  a.in = (const typename hs::cplx_t<T>::type*)c->B[in];
  a.out = (typename hs::cplx_t<T>::type*)c->B[in ^ 1];
  for (int i = 0; i < 6; ++i) a.E[i] = (T)E[i];
  a.src = src;
  if (src != nullptr) {
    a.sig0 = nullptr;
    a.Edev = nullptr;
  }
  a.skip_if_done = 1;
  const size_t sm = march_smem(c->n1, c->ty, sizeof(T) == 8, hs::MODE_FORCE, false, src != nullptr);
  LaunchScope ls(c, HS_K_XPASS);
  cudaError_t e = hs::launch_march<T>(a, c->iso, c->ty, hs::MODE_FORCE, false, c->grid_m, c->nthr_m, sm, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_march(force)");
  return HS_OK;
}

template <typename T> hs_status launch_rows(hs_ctx* c, int mode, double* acc64, bool skip) {
  hs::RowArgs<T> a;
  memset(&a, 0, sizeof(a));
  using C = typename hs::cplx_t<T>::type;
  a.spec_in = (const C*)c->B[0];
  a.spec_out = (C*)c->B[0];
  a.real_in = (const T*)c->F;
  a.real_out = acc64 ? nullptr : (T*)c->B[1];
  a.acc64 = acc64;
  a.tw = (const C*)c->twk[0];
  a.plan = c->plan[0];
  a.n1 = c->n1;
  a.P = c->P;
  a.nrows = 3 * c->n2 * c->n3;
  a.st = c->st;
  a.skip_if_done = skip ? 1 : 0;
  a.zstride = c->batch_stride;
  cudaError_t e;
  {
    LaunchScope ls(c, acc64 ? HS_K_OTHER : (mode == hs::ROW_C2R ? HS_K_XINV : HS_K_XFWD));
    e = hs::launch_row<T>(a, mode, zg(c, dim3(c->nblk_row[mode])), c->nthr_row, c->smem_row[mode], c->stream);
  }
  if (e != cudaSuccess)
    return cuda_fail(c, e, (std::string("k_row(") + (mode == hs::ROW_C2R ? "C2R" : "R2C") + ", blocks " +
                            std::to_string(c->nblk_row[mode]) + ", smem " + std::to_string(c->smem_row[mode]) + ")")
                               .c_str());
  return HS_OK;
}

// split x-pass: real-space stencil on the real displacement B[1], real force into F
template <typename T> hs_status launch_stencil(hs_ctx* c, const double E[6], const float* src, int mode, void* eps,
                                               void* sig) {
  hs::MarchArgs<T> a;
  fill_march_common<T>(c, a);
  a.ureal = (const T*)c->B[1];
  for (int i = 0; i < 6; ++i) a.E[i] = (T)E[i];
  a.src = src;
  if (src != nullptr) {  // correction equation K du = -r: linear, no eigenstrain, macro strain 0
    a.sig0 = nullptr;
    a.Edev = nullptr;
  }
  a.fout = c->F;
  a.fout_f32 = 0;
  a.eps_out = eps;
  a.sig_out = sig;
  a.out_f32 = c->opt.out_f32;
  a.skip_if_done = (mode == hs::MODE_FORCE) ? 1 : 0;
  const size_t sm = march_smem(c->n1, c->ty, sizeof(T) == 8, mode, true, src != nullptr);
  cudaError_t e;
  {
    LaunchScope ls(c, mode == hs::MODE_FORCE ? (src != nullptr ? HS_K_XPASS_SRC : HS_K_XPASS) : HS_K_FIELDS);
    e = hs::launch_march<T>(a, c->iso, c->ty, mode, true, zg(c, c->grid_m), c->nthr_m, sm, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "k_march(real)");
  return HS_OK;
}

// cuTensorMapEncodeTiled from the driver, through the runtime (null if unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// The tensor map of the column-pass tiles of B[b] (see ColArgs::tmap): T elements of the half
// spectrum as (2P x-values, 3 components, n2, n3, items) with the components' stride inside y,
// box (2 ct, 3, min(n2, 256), 1, 1) for the y passes (zax = 0) or (2 ct, 3, 1, min(n3, 256), 1)
// for the z pass (zax = 1).  Made once per buffer, base and batch shape.  False when the driver
// offers no encoder or refuses the map; the caller then copies with cp.async.
bool tile_map(hs_ctx* c, int zax, int b, CUtensorMap* out) {
  const void* base = c->B[b];
  const int n = std::max(1, c->batch_n);
  if (c->tmap_base[zax][b] != base || c->tmap_stride[zax][b] != c->batch_stride || c->tmap_n[zax][b] != n) {
    c->tmap_base[zax][b] = base;
    c->tmap_stride[zax][b] = c->batch_stride;
    c->tmap_n[zax][b] = n;
    c->tmap_ok[zax][b] = false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    const size_t cs = c->f64 ? 16 : 8;
    const size_t row = (size_t)c->P * cs, plane = row * c->n2, comp = plane * c->n3;
    const int L = zax ? c->n3 : c->n2;
    const cuuint64_t dims[5] = {(cuuint64_t)2 * c->P, 3, (cuuint64_t)c->n2, (cuuint64_t)c->n3, (cuuint64_t)n};
    const cuuint64_t strides[4] = {comp, row, plane, c->batch_stride != 0 ? c->batch_stride : 3 * comp};
    const cuuint32_t box[5] = {(cuuint32_t)(2 * c->ct), 3, zax ? 1u : (cuuint32_t)std::min(L, 256),
                               zax ? (cuuint32_t)std::min(L, 256) : 1u, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const bool aligned = ((uintptr_t)base % 16 == 0) && (2 * c->ct * (cs / 2)) % 16 == 0 && row % 16 == 0 &&
                         (c->batch_stride % 16 == 0) && (L <= 256 || L % 256 == 0);
    if (enc != nullptr && aligned &&
        enc(&c->tmap[zax][b], c->f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5,
            const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      c->tmap_ok[zax][b] = true;
  }
  if (c->tmap_ok[zax][b]) *out = c->tmap[zax][b];
  return c->tmap_ok[zax][b];
}

// ColArgs of a column pass over B[b] (zax: 0 = y passes, only where they run persistent; 1 = z
// pass, one tile per block with the state read point by point): tensor copies where the option
// and the map allow
template <typename T> hs_status set_tile_map(hs_ctx* c, hs::ColArgs<T>& a, int zax, int b) {
  a.tma = 0;
  const bool applies = zax == 0 ? c->pipe_y : !c->zstate_smem;
  if (!applies || c->opt.col_copy == 1) return HS_OK;
  if (tile_map(c, zax, b, &a.tmap)) {
    a.tma = 1;
    return HS_OK;
  }
  if (c->opt.col_copy == 2) return fail(c, HS_ERR_UNSUPPORTED_SIZE, "tensor copies unavailable for the column passes");
  return HS_OK;
}

template <typename T> hs_status launch_cols(hs_ctx* c, int buf) {
  hs::ColArgs<T> a;
  cudaError_t e;
  fill_col<T>(c, a, c->B[buf], 1);
  if (hs_status st = set_tile_map<T>(c, a, 0, buf); st != HS_OK) return st;
  {
    LaunchScope ls(c, HS_K_YFWD);
    e = c->pipe_y ? hs::launch_colp<T>(a, hs::COL_Y_FWD, c->ct, zg(c, dim3(c->nblk_py)), c->nthr_y, c->smem_py, c->stream)
                  : hs::launch_col<T>(a, hs::COL_Y_FWD, c->ct, zg(c, c->grid_y), c->nthr_y, c->smem_y, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "k_col(y fwd)");
  fill_col<T>(c, a, c->B[buf], 2);
  if (hs_status st = set_tile_map<T>(c, a, 1, buf); st != HS_OK) return st;
  {
    LaunchScope ls(c, HS_K_ZGREEN);
    e = c->pipe_z ? hs::launch_colp<T>(a, hs::COL_Z_GREEN, c->ct, zg(c, dim3(c->nblk_pz)), c->nthr_z, c->smem_pz,
                                       c->stream)
                  : hs::launch_col<T>(a, hs::COL_Z_GREEN, c->ct, zg(c, c->grid_z), c->nthr_z, c->smem_z, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "k_col(z green)");
  fill_col<T>(c, a, c->B[buf], 1);
  if (hs_status st = set_tile_map<T>(c, a, 0, buf); st != HS_OK) return st;
  {
    LaunchScope ls(c, HS_K_YINV);
    e = c->pipe_y ? hs::launch_colp<T>(a, hs::COL_Y_INV, c->ct, zg(c, dim3(c->nblk_py)), c->nthr_y, c->smem_py, c->stream)
                  : hs::launch_col<T>(a, hs::COL_Y_INV, c->ct, zg(c, c->grid_y), c->nthr_y, c->smem_y, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "k_col(y inv)");
  return HS_OK;
}

// state S -> buffer (inverse z then inverse y): the x-pass input of u = S
template <typename T> hs_status launch_state_to_buf(hs_ctx* c, int buf) {
  hs::ColArgs<T> a;
  fill_col<T>(c, a, c->B[buf], 2);
  a.skip_if_done = 0;
  cudaError_t e;
  {
    LaunchScope ls(c, HS_K_OTHER);
    e = hs::launch_col<T>(a, hs::COL_Z_INV_STATE, c->ct, zg(c, c->grid_z), c->nthr_z, c->smem_z, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "k_col(z inv state)");
  fill_col<T>(c, a, c->B[buf], 1);
  a.skip_if_done = 0;
  {
    LaunchScope ls(c, HS_K_OTHER);
    e = hs::launch_col<T>(a, hs::COL_Y_INV, c->ct, zg(c, c->grid_y), c->nthr_y, c->smem_y, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "k_col(y inv)");
  return HS_OK;
}

template <typename T> hs_status launch_fields(hs_ctx* c, const double E[6], int in, void* eps, void* sig) {
  hs::MarchArgs<T> a;
  fill_march_common<T>(c, a);
  a.in = (const typename hs::cplx_t<T>::type*)c->B[in];
  for (int i = 0; i < 6; ++i) a.E[i] = (T)E[i];
  a.eps_out = eps;
  a.sig_out = sig;
  a.out_f32 = c->opt.out_f32;
  a.skip_if_done = 0;
  const size_t sm = march_smem(c->n1, c->ty, sizeof(T) == 8, hs::MODE_FIELDS, false);
  LaunchScope ls(c, HS_K_FIELDS);
  cudaError_t e = hs::launch_march<T>(a, c->iso, c->ty, hs::MODE_FIELDS, false, c->grid_m, c->nthr_m, sm, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_march(fields)");
  return HS_OK;
}

hs_status reset_status(hs_ctx* c, double tol, int max_iter, double denom, const double* E = nullptr,
                       double rel_tol = 0.0) {
  DevStatus h;
  memset(&h, 0, sizeof(h));
  h.max_iter = max_iter;
  h.hist_cap = kHistCap;
  h.tol = tol;
  h.denom = denom;
  h.nvox = (double)c->N;
  h.macro = c->dev_macro ? c->macro : nullptr;
  h.rel_tol = rel_tol;
  for (int i = 0; i < 6; ++i) h.E[i] = E ? E[i] : c->Einit[i];
  HS_CU(c, cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  return HS_OK;
}

hs_status read_status(hs_ctx* c, DevStatus* h) {
  HS_CU(c, cudaMemcpyAsync(h, c->st, sizeof(*h), cudaMemcpyDeviceToHost, c->stream));
  HS_CU(c, cudaStreamSynchronize(c->stream));
  return HS_OK;
}

size_t cbuf_bytes(const hs_ctx* c) {
  return (size_t)3 * c->n3 * c->n2 * c->P * (c->f64 ? 16 : 8);
}

// Basic-scheme iterations until the device status says done.  Buffer c->cur
// holds the x-pass input on entry.  Returns the index of the buffer that
// holds the x-pass input of the last evaluation.
template <typename T>
hs_status iterate(hs_ctx* c, const double E[6], const float* src, DevStatus* hst, int* last_in) {
  const int cur0 = c->cur;
  int cur = cur0;
  const int chunk = std::max(1, c->opt.check_every);
  // the legacy default stream cannot be captured: plain launches there
  const bool graphs = c->opt.use_graphs && !c->xfuse && c->stream != nullptr && c->stream != cudaStreamLegacy &&
                      c->stream != cudaStreamPerThread;
  const int gi = (src != nullptr) ? 1 : 0;
  ChunkProfGuard guard{c};
  for (;;) {
    // profiling: one chunk in prof_every runs as plain launches that record kernel events;
    // the others run as they would without profiling
    const bool sampled = c->prof && (c->chunk_seq++ % c->prof_every) == 0;
    c->prof_skip = c->prof && !sampled;
    if (graphs && !sampled && c->gexec[gi] != nullptr) {
      HS_CU(c, cudaGraphLaunch(c->gexec[gi], c->stream));
      account_replay(c, gi);
      hs_status s = read_status(c, hst);
      if (s != HS_OK) return s;
      if (hst->done) break;
      continue;
    }
    bool capture = graphs && !sampled && c->gchunks[gi] >= 1;
    if (capture) {
      drop_graph(c, gi, false);
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        // a stream that refuses capture (e.g. one already being captured): plain launches from now on
        cudaGetLastError();
        c->opt.use_graphs = 0;
        capture = false;
      }
    }
    if (capture) {
      c->capturing = true;
      c->cap_gi = gi;
    }
    for (int i = 0; i < chunk; ++i) {
      if (c->xfuse) {
        hs_status s = launch_force<T>(c, E, cur, src);
        if (s != HS_OK) return s;
        s = launch_cols<T>(c, cur ^ 1);
        if (s != HS_OK) return s;
        cur ^= 1;
      } else {
        hs_status s = launch_rows<T>(c, hs::ROW_C2R, nullptr, true);
        if (s == HS_OK) s = launch_stencil<T>(c, E, src, hs::MODE_FORCE, nullptr, nullptr);
        if (s == HS_OK) s = launch_rows<T>(c, hs::ROW_R2C, nullptr, true);
        if (s == HS_OK) s = launch_cols<T>(c, 0);
        if (s != HS_OK) {
          if (capture) {
            c->capturing = false;
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(c->stream, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            drop_graph(c, gi, false);
          }
          return s;
        }
      }
    }
    if (capture) {
      // the captured chunk has not run yet: instantiate it, keep it, and launch it
      c->capturing = false;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      cudaGraphExec_t ex = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        drop_graph(c, gi, false);
        return cuda_fail(c, e, "graph capture");
      }
      c->gexec[gi] = ex;
      HS_CU(c, cudaGraphLaunch(ex, c->stream));
      account_replay(c, gi);
    }
    ++c->gchunks[gi];
    hs_status s = read_status(c, hst);
    if (s != HS_OK) return s;
    if (hst->done) break;
  }
  *last_in = c->xfuse ? (cur0 ^ ((hst->evals - 1) & 1)) : 0;
  return HS_OK;
}

hs_status status_code(const DevStatus& h) {
  if (h.done == hs::DONE_TIMEOUT) return HS_ERR_TIMEOUT;
  if (h.done == hs::DONE_FAULT) return HS_ERR_CUDA;
  if (h.done == hs::DONE_CONVERGED) return HS_OK;
  if (h.done == hs::DONE_DIVERGED) return HS_DIVERGED;
  return HS_NOT_CONVERGED;
}

template <typename T>
hs_status solve_plain(hs_ctx* c, const double E[6], double tol, int max_iter, void* eps, void* sig,
                      double sig_eff[6], int* iters, double* final_err, double* E_final) {
  hs_status s = reset_status(c, tol, max_iter, 0.0, c->dev_macro ? nullptr : E);
  if (s != HS_OK) return s;
  c->cur = 0;
  if (c->warm) {
    s = launch_state_to_buf<T>(c, 0);
    if (s != HS_OK) return s;
    c->warm = false;
  } else {
    HS_CU(c, cudaMemsetAsync(c->S, 0, cbuf_bytes(c), c->stream));
    HS_CU(c, cudaMemsetAsync(c->B[0], 0, cbuf_bytes(c), c->stream));
  }
  DevStatus h;
  int last_in = 0;
  s = iterate<T>(c, E, nullptr, &h, &last_in);
  if (s != HS_OK) return s;
  if (eps != nullptr && sig != nullptr) {
    if (c->xfuse) {
      s = launch_fields<T>(c, E, last_in, eps, sig);
    } else {
      s = launch_rows<T>(c, hs::ROW_C2R, nullptr, false);
      if (s == HS_OK) s = launch_stencil<T>(c, E, nullptr, hs::MODE_FIELDS, eps, sig);
    }
    if (s != HS_OK) return s;
  }
  HS_CU(c, cudaStreamSynchronize(c->stream));
  const int n = std::min(h.evals, kHistCap);
  c->hist_host.resize(n);
  if (n) HS_CU(c, cudaMemcpy(c->hist_host.data(), c->hist, n * sizeof(double), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 6; ++i) sig_eff[i] = h.sig_mean[i];
  if (E_final) for (int i = 0; i < 6; ++i) E_final[i] = c->dev_macro ? h.E[i] : E[i];
  if (iters) *iters = h.evals;
  if (final_err) *final_err = h.err;
  return status_code(h);
}

// FP64 real-space residual sweep on u64: force -> rsrc (float), status -> err
hs_status launch_residual64(hs_ctx* c, const double E[6], int mode, void* eps, void* sig) {
  hs::MarchArgs<double> a;
  fill_march_common<double>(c, a);
  a.mat = c->matd;
  for (int i = 0; i < 6; ++i) a.E[i] = E[i];
  a.ureal = c->u64;
  a.fout = c->rsrc;
  a.fout_f32 = 1;
  a.zc = c->zc64;
  a.eps_out = eps;
  a.sig_out = sig;
  a.out_f32 = c->opt.out_f32;
  a.skip_if_done = 0;
  const size_t sm = march_smem(c->n1, c->ty64, true, mode, true);
  LaunchScope ls(c, mode == hs::MODE_FIELDS ? HS_K_FIELDS : HS_K_RESID64);
  cudaError_t e = hs::launch_march<double>(a, c->iso, c->ty64, mode, true, zg(c, c->grid_m64), c->nthr_m, sm, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_march(residual fp64)");
  return HS_OK;
}

hs_status launch_emit(hs_ctx* c, int in) {
  hs::MarchArgs<float> a;
  fill_march_common<float>(c, a);
  a.in = (const float2*)c->B[in];
  a.u64 = c->u64;
  a.skip_if_done = 0;
  const size_t sm = march_smem(c->n1, c->ty, false, hs::MODE_EMIT, false);
  LaunchScope ls(c, HS_K_OTHER);
  cudaError_t e = hs::launch_march<float>(a, true, c->ty, hs::MODE_EMIT, false, c->grid_m, c->nthr_m, sm, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_march(emit)");
  return HS_OK;
}

// Frobenius norm of a Voigt-ordered symmetric tensor (shear entries counted twice)
double frob(const double v[6]) {
  double s = 0;
  for (int i = 0; i < 6; ++i) s += (i < 3 ? 1.0 : 2.0) * v[i] * v[i];
  return std::sqrt(s);
}

// Sa != nullptr: applied-stress control.  The FP64 sweeps use the current
// macroscopic strain; after a sweep that does not stop, E <- E + S0 (sigma^a -
// <sigma>) (Algorithm 1 step 6, regrouped), and stopping also needs
// ||sigma^a - <sigma>|| < tol max(||sigma^a||, ||<sigma>||): the correction
// solves restore equilibrium for a given E long before E settles.
hs_status solve_refined(hs_ctx* c, const double E0[6], double tol, int max_iter, void* eps, void* sig,
                        double sig_eff[6], int* iters, double* final_err, const double* Sa, const double* S0,
                        double* E_final) {
  double E[6];
  for (int i = 0; i < 6; ++i) E[i] = E0[i];
  HS_CU(c, cudaMemsetAsync(c->u64, 0, 3 * c->N * sizeof(double), c->stream));
  c->hist_host.clear();
  int total = 0;
  DevStatus h64, hin;
  const double zeroE[6] = {0, 0, 0, 0, 0, 0};
  hs_status result = HS_NOT_CONVERGED;
  // At u64 = 0 the correction equation is the problem itself: its first FP32
  // solve is the plain basic scheme under E (and the eigenstrain), run until
  // its error falls to inner_ratio times its first error, so no FP64 sweep is
  // spent on the residual of the zero displacement.  Every stop decision is
  // still taken on an FP64 sweep.
  if (max_iter > 1) {
    const int budget = std::min(std::max(1, c->opt.inner_max), max_iter - 1);
    hs_status s = reset_status(c, 0.0, budget, 0.0, E, c->opt.inner_ratio);
    if (s != HS_OK) return s;
    HS_CU(c, cudaMemsetAsync(c->S, 0, cbuf_bytes(c), c->stream));
    HS_CU(c, cudaMemsetAsync(c->B[0], 0, cbuf_bytes(c), c->stream));
    c->cur = 0;
    int last_in = 0;
    s = iterate<float>(c, E, nullptr, &hin, &last_in);
    if (s != HS_OK) return s;
    total += hin.evals;
    {
      const int n = std::min(hin.evals, kHistCap);
      std::vector<double> h32(n);
      if (n) HS_CU(c, cudaMemcpy(h32.data(), c->hist, n * sizeof(double), cudaMemcpyDeviceToHost));
      c->hist_host.insert(c->hist_host.end(), h32.begin(), h32.end());
    }
    if (hin.done == hs::DONE_TIMEOUT) return fail(c, HS_ERR_TIMEOUT, "a bounded device wait gave up");
    if (hin.done == hs::DONE_FAULT) return fail(c, HS_ERR_CUDA, "a kernel's alignment check failed");
    if (hin.done == hs::DONE_DIVERGED) {
      HS_CU(c, cudaStreamSynchronize(c->stream));
      for (int i = 0; i < 6; ++i) sig_eff[i] = hin.sig_mean[i];
      if (E_final) for (int i = 0; i < 6; ++i) E_final[i] = E[i];
      if (iters) *iters = total;
      if (final_err) *final_err = hin.err;
      return HS_DIVERGED;
    }
    s = launch_state_to_buf<float>(c, 0);
    if (s != HS_OK) return s;
    s = c->xfuse ? launch_emit(c, 0) : launch_rows<float>(c, hs::ROW_C2R, c->u64, false);
    if (s != HS_OK) return s;
  }
  bool fields_done = false;
  for (;;) {
    hs_status s = reset_status(c, 0.0, 1 << 30, 0.0, E);
    if (s != HS_OK) return s;
    // a sweep that uses up the evaluation budget is the last: it also writes the fields
    const bool last = (total + 1 >= max_iter) && eps != nullptr && sig != nullptr;
    s = last ? launch_residual64(c, E, hs::MODE_FORCE_FIELDS, eps, sig)
             : launch_residual64(c, E, hs::MODE_FORCE, nullptr, nullptr);
    fields_done = last;
    if (s != HS_OK) return s;
    s = read_status(c, &h64);
    if (s != HS_OK) return s;
    total += 1;
    c->hist_host.push_back(h64.err);
    if (!(h64.err == h64.err) || h64.err > 1e300) { result = HS_DIVERGED; break; }
    bool stress_ok = true;
    if (Sa != nullptr) {
      double d[6];
      for (int i = 0; i < 6; ++i) d[i] = Sa[i] - h64.sig_mean[i];
      const double den = std::max({frob(Sa), frob(h64.sig_mean), 1e-300});
      stress_ok = frob(d) < tol * den;
    }
    if (h64.err < tol && stress_ok) { result = HS_OK; break; }
    if (total >= max_iter) { result = HS_NOT_CONVERGED; break; }
    if (Sa != nullptr) {
      for (int i = 0; i < 6; ++i) {
        double acc = 0;
        for (int j = 0; j < 6; ++j) acc += S0[i * 6 + j] * (Sa[j] - h64.sig_mean[j]);
        E[i] += acc;
      }
    }
    // correction solve: K du = -r in FP32, source r = rsrc, macro strain 0
    const int budget = std::min(std::max(1, c->opt.inner_max), max_iter - total);
    s = reset_status(c, c->opt.inner_ratio * h64.err, budget, h64.sig_norm, zeroE);
    if (s != HS_OK) return s;
    HS_CU(c, cudaMemsetAsync(c->S, 0, cbuf_bytes(c), c->stream));
    HS_CU(c, cudaMemsetAsync(c->B[0], 0, cbuf_bytes(c), c->stream));
    c->cur = 0;
    int last_in = 0;
    s = iterate<float>(c, zeroE, c->rsrc, &hin, &last_in);
    if (s != HS_OK) return s;
    total += hin.evals;
    if (hin.done == hs::DONE_TIMEOUT) return fail(c, HS_ERR_TIMEOUT, "a bounded device wait gave up");
    if (hin.done == hs::DONE_FAULT) return fail(c, HS_ERR_CUDA, "a kernel's alignment check failed");
    if (hin.done == hs::DONE_DIVERGED) { result = HS_DIVERGED; break; }
    // u64 += du, du = inverse transform of the correction state
    s = launch_state_to_buf<float>(c, 0);
    if (s != HS_OK) return s;
    s = c->xfuse ? launch_emit(c, 0) : launch_rows<float>(c, hs::ROW_C2R, c->u64, false);
    if (s != HS_OK) return s;
  }
  if (eps != nullptr && sig != nullptr && !fields_done) {
    hs_status s = launch_residual64(c, E, hs::MODE_FIELDS, eps, sig);
    if (s != HS_OK) return s;
  }
  HS_CU(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < 6; ++i) sig_eff[i] = h64.sig_mean[i];
  if (E_final) for (int i = 0; i < 6; ++i) E_final[i] = E[i];
  if (iters) *iters = total;
  if (final_err) *final_err = h64.err;
  return result;
}

// 6x6 inverse by Gauss-Jordan elimination with partial pivoting; false if singular
bool inv6(const double A[36], double X[36]) {
  double M[6][12];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 12; ++j) M[i][j] = j < 6 ? A[i * 6 + j] : (j - 6 == i ? 1.0 : 0.0);
  double scale = 0;
  for (int i = 0; i < 36; ++i) scale = std::max(scale, std::fabs(A[i]));
  for (int col = 0; col < 6; ++col) {
    int piv = col;
    for (int r = col + 1; r < 6; ++r)
      if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
    if (!(std::fabs(M[piv][col]) > 1e-14 * scale)) return false;
    if (piv != col)
      for (int j = 0; j < 12; ++j) std::swap(M[piv][j], M[col][j]);
    const double d = M[col][col];
    for (int j = 0; j < 12; ++j) M[col][j] /= d;
    for (int r = 0; r < 6; ++r) {
      if (r == col) continue;
      const double f = M[r][col];
      if (f != 0)
        for (int j = 0; j < 12; ++j) M[r][j] -= f * M[col][j];
    }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) X[i * 6 + j] = M[i][j + 6];
  return true;
}

}  // namespace

extern "C" {

hs_status hs_default_options(hs_options* opt) {
  if (!opt) return HS_ERR_INVALID_ARG;
  opt->precision = HS_FP64;
  opt->check_every = 8;
  opt->out_f32 = 0;
  opt->inner_max = 200;
  opt->inner_ratio = 1e-3;
  opt->zchunk = 0;
  opt->ytile = 0;
  opt->xfuse = 0;
  opt->col_tile = 0;
  opt->col_threads = 0;
  opt->use_graphs = 1;
  opt->col_state = 0;
  opt->col_pipe = 0;
  opt->col_copy = 0;
  return HS_OK;
}

hs_status hs_workspace_size(const int grid[3], int nphase, const hs_options* opt, size_t* bytes) {
  if (!grid || !bytes || nphase < 1 || nphase > 65536) return fail(nullptr, HS_ERR_INVALID_ARG, "bad argument");
  hs_options o;
  hs_default_options(&o);
  if (opt) o = *opt;
  if (o.precision < HS_FP64 || o.precision > HS_FP32_REFINED) return fail(nullptr, HS_ERR_INVALID_ARG, "bad precision");
  hs_status s = check_grid(grid);
  if (s != HS_OK) return fail(nullptr, s, "unsupported grid size");
  *bytes = make_layout(grid[0], grid[1], grid[2], nphase, o.precision).total;
  return HS_OK;
}

// hs_create with the phase count that sizes the workspace layout given separately
// (layout_np >= m->nphase; 0: m->nphase): the items of a batched class share one
// layout, so each is created with the largest phase count of its class.
static hs_status create_impl(hs_ctx** out, const int grid[3], const hs_material* m_in, const double C0[36],
                             const hs_options* opt, void* workspace, size_t workspace_bytes, void* stream,
                             int layout_np) {
  if (!out || !grid || !m_in || !workspace) return fail(nullptr, HS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (m_in->kind == HS_COEFFS_F32) {
    hs_status sg = check_grid(grid);
    if (sg != HS_OK) return fail(nullptr, sg, "unsupported grid size");
  }
  IdsMaterial im;
  {
    hs_status sm = to_ids_material(m_in, grid, stream, &im);
    if (sm == HS_ERR_CUDA) return fail(nullptr, sm, g_last_error);
    if (sm == HS_ERR_UNSUPPORTED_SIZE)
      return fail(nullptr, sm, "more than HS_MAX_PHASES distinct stiffnesses in the per-voxel field");
    if (sm != HS_OK) return fail(nullptr, sm, "bad per-voxel stiffness field (null or non-finite)");
  }
  const hs_material* m = im.use;
  if (!m->ids || !m->table) return fail(nullptr, HS_ERR_INVALID_ARG, "null argument");
  hs_options o;
  hs_default_options(&o);
  if (opt) o = *opt;
  if (o.precision < HS_FP64 || o.precision > HS_FP32_REFINED || o.check_every < 1 || o.inner_max < 1 ||
      !(o.inner_ratio > 0 && o.inner_ratio < 1) || o.zchunk < 0 ||
      !(o.ytile == 0 || ((o.ytile == 2 || o.ytile == 4 || o.ytile == 8) && grid[1] % o.ytile == 0)) ||
      (o.xfuse != 0 && o.xfuse != 1) || o.col_tile < 0 || o.col_threads < 0 || (o.col_threads % 32) != 0 ||
      (o.use_graphs != 0 && o.use_graphs != 1) || o.col_state < 0 || o.col_state > 2 ||
      o.col_pipe < 0 || o.col_pipe > 2 || o.col_copy < 0 || o.col_copy > 2)
    return fail(nullptr, HS_ERR_INVALID_ARG, "bad options");
  if (m->kind != HS_IDS_U8 && m->kind != HS_IDS_U16) return fail(nullptr, HS_ERR_INVALID_ARG, "bad id kind");
  if (m->nphase < 1 || m->nphase > HS_MAX_PHASES)
    return fail(nullptr, HS_ERR_INVALID_ARG, "bad nphase");
  hs_status s = check_grid(grid);
  if (s != HS_OK) return fail(nullptr, s, "unsupported grid size (even, 4..512, prime factors 2, 3, 5, 7, 11)");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(nullptr, HS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  // material table checks
  const int np = m->nphase;
  std::vector<double> table(m->table, m->table + (size_t)np * 36);
  bool all_iso = true;
  std::vector<double> lam(np), mu(np);
  for (int p = 0; p < np; ++p) {
    const double* C = &table[(size_t)p * 36];
    double scale = 0;
    for (int i = 0; i < 36; ++i) {
      if (!std::isfinite(C[i])) return fail(nullptr, HS_ERR_INVALID_ARG, "non-finite stiffness");
      scale = std::max(scale, fabs(C[i]));
    }
    for (int i = 0; i < 6; ++i) {
      if (C[i * 6 + i] < 0) return fail(nullptr, HS_ERR_INVALID_ARG, "negative stiffness diagonal");
      for (int j = 0; j < i; ++j)
        if (fabs(C[i * 6 + j] - C[j * 6 + i]) > 1e-12 * scale)
          return fail(nullptr, HS_ERR_INVALID_ARG, "stiffness table not symmetric");
    }
    if (!is_isotropic(C, &lam[p], &mu[p])) all_iso = false;
  }
  // reference medium
  double C0v[36];
  if (C0) {
    for (int i = 0; i < 36; ++i) C0v[i] = C0[i];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < i; ++j)
        if (fabs(C0v[i * 6 + j] - C0v[j * 6 + i]) > 1e-12 * fabs(C0v[0]))
          return fail(nullptr, HS_ERR_INVALID_ARG, "C0 not symmetric");
    if (!cholesky_pd(C0v)) return fail(nullptr, HS_ERR_INVALID_ARG, "C0 not positive definite");
  } else if (np == 2 && all_iso) {
    // Section 3.4: same Poisson ratio, k0 = alpha k_m + (1 - alpha) k_i
    const double km = lam[0] + 2 * mu[0] / 3, ki = lam[1] + 2 * mu[1] / 3;
    const double alpha = (ki < km) ? 0.55 : 0.45;
    const double k0 = alpha * km + (1 - alpha) * ki;
    const double nu0 = lam[0] / (2 * (lam[0] + mu[0]));
    const double mu0 = 3 * k0 * (1 - 2 * nu0) / (2 * (1 + nu0));
    iso_voigt(k0 - 2 * mu0 / 3, mu0, C0v);
    if (!cholesky_pd(C0v)) return fail(nullptr, HS_ERR_INVALID_ARG, "reference medium not positive definite");
  } else {
    double kmin = 1e300, kmax = -1e300, dmin = 1e300, dmax = -1e300;
    for (int p = 0; p < np; ++p) {
      double K, d0, d1;
      bulk_and_shear_range(&table[(size_t)p * 36], &K, &d0, &d1);
      kmin = std::min(kmin, K);
      kmax = std::max(kmax, K);
      dmin = std::min(dmin, d0);
      dmax = std::max(dmax, d1);
    }
    const double k0 = 0.5 * (kmin + kmax), mu0 = 0.25 * (dmin + dmax);
    iso_voigt(k0 - 2 * mu0 / 3, mu0, C0v);
    if (!cholesky_pd(C0v)) return fail(nullptr, HS_ERR_INVALID_ARG, "reference medium not positive definite");
  }

  hs_ctx* c = new hs_ctx();
  {
    double l0 = 0, m0 = 0;
    c->c0_iso = is_isotropic(C0v, &l0, &m0);
    c->c0_a = l0 + m0;
    c->c0_b = m0;
  }
  c->n1 = grid[0];
  c->n2 = grid[1];
  c->n3 = grid[2];
  c->nh = c->n1 / 2 + 1;
  c->prec = o.precision;
  c->f64 = (o.precision == HS_FP64);
  c->P = pitch_of(c->nh, c->f64);
  c->N = (size_t)c->n1 * c->n2 * c->n3;
  c->opt = o;
  c->stream = (cudaStream_t)stream;
  c->nphase = np;
  c->iso = all_iso;
  c->table = table;
  memcpy(c->C0, C0v, sizeof(C0v));
  // Omega^-1_jl = sum_ik lambda0_jikl M_ik, M symmetric: G6[(j,l)][(i,k)]
  static const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      const int j = pr[a][0], l = pr[a][1], i = pr[b][0], k = pr[b][1];
      double g = C0v[vidx(j, i) * 6 + vidx(k, l)];
      if (i != k) g += C0v[vidx(j, k) * 6 + vidx(i, l)];
      c->G6[a * 6 + b] = g;
    }
  c->layout_np = std::max(np, layout_np);
  c->lay = make_layout(c->n1, c->n2, c->n3, c->layout_np, o.precision);
  if (workspace_bytes < c->lay.total) {
    delete c;
    return fail(nullptr, HS_ERR_OOM, "workspace too small");
  }
  c->ws = (char*)workspace;
  c->ws_bytes = workspace_bytes;
  c->S = c->ws + c->lay.S;
  c->B[0] = c->ws + c->lay.B0;
  c->B[1] = c->ws + c->lay.B1;
  c->F = c->ws + c->lay.F;
  c->ids = (uint16_t*)(c->ws + c->lay.ids);
  c->matk = c->ws + c->lay.matk;
  c->matd = (double*)(c->ws + c->lay.matd);
  c->partials = (double*)(c->ws + c->lay.partials);
  c->st = (DevStatus*)(c->ws + c->lay.status);
  c->hist = (double*)(c->ws + c->lay.hist);
  c->macro = (double*)(c->ws + c->lay.macro);
  c->sig0f = (float*)(c->ws + c->lay.sig0f);
  c->sig0d = (double*)(c->ws + c->lay.sig0d);
  c->u64 = (o.precision == HS_FP32_REFINED) ? (double*)(c->ws + c->lay.u64) : nullptr;
  c->rsrc = (o.precision == HS_FP32_REFINED) ? (float*)(c->ws + c->lay.rsrc) : nullptr;
  c->warm = false;
  c->cur = 0;
  c->prof = false;
  for (int k = 0; k < HS_K_COUNT; ++k) c->launches[k] = 0;
  for (int ax = 0; ax < 3; ++ax) make_plan(grid[ax], &c->plan[ax]);

  // launch configuration
  c->ty = o.ytile > 0 ? o.ytile : pick_ty(c->n2);
  c->nthr_m = ((c->n1 + 31) / 32) * 32;
  const int ytiles = c->n2 / c->ty;
  int nzc = std::max(1, std::min(c->n3, (kTargetBlocks + ytiles - 1) / ytiles));
  c->zc = (c->n3 + nzc - 1) / nzc;
  if (o.zchunk > 0) c->zc = std::min(o.zchunk, c->n3);
  nzc = (c->n3 + c->zc - 1) / c->zc;
  c->grid_m = dim3(ytiles, nzc);
  // measured on GB300 at 256^3: narrow tiles in small blocks overlap best
  // (compile-time y/z kernels: 256 threads 0.096 / 0.218 ms, 768 threads
  // 0.115 / 0.235 ms per y / z+Green pass)
  c->ct = c->f64 ? 4 : 8;
  if (o.col_tile > 0) {
    if (o.col_tile != (c->f64 ? 8 : 16) && o.col_tile != (c->f64 ? 4 : 8)) {
      delete c;
      return fail(nullptr, HS_ERR_INVALID_ARG, "col_tile must be 8 or 16 (FP32), 4 or 8 (FP64)");
    }
    c->ct = o.col_tile;
  }
  const int maxthr = c->f64 ? 384 : 768;
  if (o.col_threads > maxthr) {
    delete c;
    return fail(nullptr, HS_ERR_INVALID_ARG, "col_threads above the block limit");
  }
  auto col_threads = [&](int L) {
    const int T = (L + hs::kE - 1) / hs::kE;
    int n = 3 * c->ct * T;
    n = ((n + 31) / 32) * 32;
    n = std::min(n, (maxthr / T) * T);
    const int dflt = c->f64 ? 128 : 256;
    n = std::min(n, std::max(T, (dflt / T) * T));
    if (o.col_threads > 0) n = std::max(T, (o.col_threads / T) * T);
    return n;
  };
  c->nthr_y = col_threads(c->n2);
  c->nthr_z = col_threads(c->n3);
  const size_t cs = c->f64 ? 16 : 8;
  // a tile, then (fixed lengths) the twiddle table 16 bytes behind it
  c->smem_y = (size_t)c->n2 * 3 * c->ct * cs + 16 + (size_t)c->n2 * cs;
  // the z pass may load its tile by a tensor copy: room for its alignment and barrier
  c->smem_z = (size_t)c->n3 * 3 * c->ct * cs + hs::kColpTmaSlack + 2 * (size_t)c->n3 * cs;
  c->xfuse = (o.xfuse == 1);
  {
    // radix-5/7/11 lengths run the split path with the default column tile only
    const bool ext = hs::plan_ext(c->plan[0]) || hs::plan_ext(c->plan[1]) || hs::plan_ext(c->plan[2]);
    if (ext && (c->xfuse || c->ct != (c->f64 ? 4 : 8))) {
      delete c;
      return fail(nullptr, HS_ERR_UNSUPPORTED_SIZE,
                  "grids with a factor 5, 7 or 11 need xfuse = 0 and the default column tile");
    }
  }
  c->nthr_row = 256;
  for (int m = 0; m < 2; ++m) c->smem_row[m] = hs::row_layout(m, c->n1, c->P, c->nthr_row, c->f64 ? 8 : 4).total;
  const int xtiles = (c->nh + c->ct - 1) / c->ct;
  c->grid_y = dim3(xtiles, c->n3);
  c->grid_z = dim3(xtiles, c->n2);
  // shared memory limits
  int dev = 0, smem_optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    hs_status st = cuda_fail(nullptr, e, "device query");
    delete c;
    return st;
  }
  // real-space pass: an automatic row tile is halved while its plane ring does not fit
  // (FP64 rows of 512 need 2 rows per block)
  if (o.ytile == 0 && !c->xfuse) {
    int ty = c->ty;
    while (ty > 2 && march_smem(c->n1, ty, c->f64, hs::MODE_FORCE, true, true) > (size_t)smem_optin) ty /= 2;
    if (ty != c->ty && c->n2 % ty == 0) {
      c->ty = ty;
      const int yt = c->n2 / c->ty;
      int nz = std::max(1, std::min(c->n3, (kTargetBlocks + yt - 1) / yt));
      c->zc = (c->n3 + nz - 1) / nz;
      if (o.zchunk > 0) c->zc = std::min(o.zchunk, c->n3);
      nz = (c->n3 + c->zc - 1) / c->zc;
      c->grid_m = dim3(yt, nz);
    }
  }
  // FP64 precision: the real-space pass is FP64-bound like the refined mode's sweep
  if (c->f64 && !c->xfuse && o.zchunk == 0) {
    int per_sm = 0, nsm = 0;
    const size_t smf = march_smem(c->n1, c->ty, true, hs::MODE_FORCE, true);
    if (hs::march_blocks_per_sm<double>(c->iso, c->ty, c->nthr_m, smf, &per_sm) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && per_sm > 0) {
      const int yt = c->n2 / c->ty;
      c->zc = pick_zchunk64(yt, c->n3, per_sm * nsm);
      c->grid_m = dim3(yt, (c->n3 + c->zc - 1) / c->zc);
    } else {
      cudaGetLastError();
    }
  }
  // FP64 residual sweep: the widest row tile whose plane ring fits; 8 rows (1/8 of the rows
  // recomputed, not 1/4, and no register spills in blocks of at most 256 threads) where N1 <= 256
  c->ty64 = c->ty;
  if (o.precision == HS_FP32_REFINED) {
    if (o.ytile == 0 && c->n1 <= 256 && c->n2 % 8 == 0 &&
        march_smem(c->n1, 8, true, hs::MODE_FORCE, true) <= (size_t)smem_optin)
      c->ty64 = 8;
    while (c->ty64 > 2 && march_smem(c->n1, c->ty64, true, hs::MODE_FORCE, true) > (size_t)smem_optin) c->ty64 /= 2;
    if (c->n2 % c->ty64 != 0) c->ty64 = 2;
  }
  {
    const int yt = c->n2 / c->ty64;
    int nz = std::max(1, std::min(c->n3, (kTargetBlocks + yt - 1) / yt));
    c->zc64 = (c->n3 + nz - 1) / nz;
    if (o.precision == HS_FP32_REFINED) {
      int per_sm = 0, nsm = 0;
      const size_t sm64 = march_smem(c->n1, c->ty64, true, hs::MODE_FORCE, true);
      if (hs::march_blocks_per_sm<double>(c->iso, c->ty64, c->nthr_m, sm64, &per_sm) == cudaSuccess &&
          cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && per_sm > 0)
        c->zc64 = pick_zchunk64(yt, c->n3, per_sm * nsm);
      else
        cudaGetLastError();
    }
    nz = (c->n3 + c->zc64 - 1) / c->zc64;
    c->grid_m64 = dim3(yt, nz);
  }
  // z pass: the state tile in shared memory beside the force tile when asked for (col_state = 2)
  if (o.col_state == 2 && 2 * c->smem_z <= (size_t)smem_optin) {
    c->zstate_smem = true;
    c->smem_z *= 2;
  }
  const size_t need = std::max({c->xfuse ? march_smem(c->n1, c->ty, c->f64, hs::MODE_FORCE, false, true)
                                          : march_smem(c->n1, c->ty, c->f64, hs::MODE_FORCE, true, true),
                                c->smem_row[0], c->smem_row[1],
                                o.precision == HS_FP32_REFINED ? march_smem(c->n1, c->ty64, true, hs::MODE_FORCE, true) : 0,
                                c->smem_y, c->smem_z});
  if (need > (size_t)smem_optin) {
    delete c;
    return fail(nullptr, HS_ERR_UNSUPPORTED_SIZE, "grid too large for shared-memory tiles");
  }
  // persistent row passes: as many blocks as stay resident, at most one per batch
  {
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int T8 = (c->n1 + hs::kE - 1) / hs::kE;
    const size_t G = (size_t)(c->nthr_row / T8);
    const size_t nbatch = ((size_t)3 * c->n2 * c->n3 / 2 + G - 1) / G;
    for (int m = 0; m < 2 && e == cudaSuccess; ++m) {
      int per_sm = 0;
      e = c->f64 ? hs::row_blocks_per_sm<double>(m, c->n1, c->nthr_row, c->smem_row[m], &per_sm)
                 : hs::row_blocks_per_sm<float>(m, c->n1, c->nthr_row, c->smem_row[m], &per_sm);
      c->nblk_row[m] = (int)std::min<size_t>(nbatch, (size_t)std::max(1, per_sm) * std::max(1, nsm));
    }
    if (e != cudaSuccess) {
      hs_status st = cuda_fail(nullptr, e, "row pass occupancy");
      delete c;
      return st;
    }
  }

  // persistent double-buffered y / z passes at the compile-time lengths (default tile and block)
  {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const bool ext = hs::plan_ext(c->plan[1]) || hs::plan_ext(c->plan[2]);
    const int xtiles = (c->nh + c->ct - 1) / c->ct;
    // the z pass stays one tile per block: its Green step waits on the state point by point, and
    // three resident blocks hide that better than two persistent ones (256^3 FP32: 0.228 against
    // 0.247 ms; the y passes gain, 0.095 against 0.101 ms)
    for (int axis = 1; axis <= (o.col_pipe == 2 ? 2 : 1) && o.col_pipe != 1 && !ext && nsm > 0; ++axis) {
      const int L = axis == 1 ? c->n2 : c->n3;
      if (L != 128 && L != 256 && L != 512) continue;
      if (axis == 2 && c->zstate_smem) continue;  // the persistent z pass reads the state point by point
      // the tiles may arrive by tensor copies: room for their alignment and barriers
      // and for the twiddle tables behind them
      const size_t smem = 2 * (size_t)L * 3 * c->ct * cs + hs::kColpTmaSlack + 2 * (size_t)L * cs;
      if (smem > (size_t)smem_optin) continue;
      const int nthr = axis == 1 ? c->nthr_y : c->nthr_z;
      int per_sm = 0;
      cudaError_t q = c->f64 ? hs::colp_blocks_per_sm<double>(axis == 1 ? hs::COL_Y_FWD : hs::COL_Z_GREEN, L, c->ct, nthr,
                                                              smem, &per_sm)
                             : hs::colp_blocks_per_sm<float>(axis == 1 ? hs::COL_Y_FWD : hs::COL_Z_GREEN, L, c->ct, nthr,
                                                             smem, &per_sm);
      if (q != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        continue;
      }
      const size_t ntiles = (size_t)xtiles * (axis == 1 ? c->n3 : c->n2);
      const int nb = (int)std::min<size_t>(ntiles, (size_t)per_sm * nsm);
      if (axis == 1) {
        c->pipe_y = true;
        c->nblk_py = nb;
        c->smem_py = smem;
      } else {
        c->pipe_z = true;
        c->nblk_pz = nb;
        c->smem_pz = smem;
      }
    }
  }

  // twiddles / phase tables in kernel precision
  {
    std::vector<double> tw;
    for (int ax = 0; ax < 3; ++ax) {
      std::vector<double> re, im;
      twiddles(grid[ax], re, im);
      for (int j = 0; j < grid[ax]; ++j) {
        tw.push_back(re[j]);
        tw.push_back(im[j]);
      }
    }
    char* twp = c->ws + c->lay.tw;
    size_t off = 0;
    for (int ax = 0; ax < 3; ++ax) {
      c->twk[ax] = twp + off;
      off += (size_t)grid[ax] * cs;
    }
    if (c->f64) {
      e = cudaMemcpyAsync(twp, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice, c->stream);
    } else {
      std::vector<float> twf(tw.begin(), tw.end());
      e = cudaMemcpyAsync(twp, twf.data(), twf.size() * 4, cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      hs_status st = cuda_fail(nullptr, e, "twiddle upload");
      delete c;
      return st;
    }
    std::vector<double> md((size_t)np * 21);
    for (int p = 0; p < np; ++p) {
      const double* C = &table[(size_t)p * 36];
      if (all_iso) {
        md[(size_t)p * 2] = lam[p];
        md[(size_t)p * 2 + 1] = mu[p];
      } else {
        int k = 0;
        for (int i = 0; i < 6; ++i)
          for (int j = i; j < 6; ++j) md[(size_t)p * 21 + k++] = C[i * 6 + j];
      }
    }
    {
      // isotropic reference medium for the Green step of batched launches: (lambda0 + mu0, mu0)
      // in FP64, then in FP32
      static_assert(sizeof(float) * 2 + sizeof(double) * 2 <= 32, "c0 region");
      unsigned char c0b[32] = {0};
      const double cd[2] = {c->c0_a, c->c0_b};
      const float cf[2] = {(float)c->c0_a, (float)c->c0_b};
      memcpy(c0b, cd, sizeof(cd));
      memcpy(c0b + 16, cf, sizeof(cf));
      e = cudaMemcpyAsync(c->ws + c->lay.c0, c0b, sizeof(c0b), cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->matd, md.data(), md.size() * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
      if (c->f64) {
        e = cudaMemcpyAsync(c->matk, md.data(), md.size() * 8, cudaMemcpyHostToDevice, c->stream);
      } else {
        std::vector<float> mf(md.begin(), md.end());
        e = cudaMemcpyAsync(c->matk, mf.data(), mf.size() * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      hs_status st = cuda_fail(nullptr, e, "material upload");
      delete c;
      return st;
    }
  }
  // phase ids (host or device pointer), converted to uint16 on the device
  {
    cudaPointerAttributes attr;
    e = cudaPointerGetAttributes(&attr, m->ids);
    bool dev_ptr = (e == cudaSuccess) && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    if (e != cudaSuccess) cudaGetLastError();
    const cudaMemcpyKind kind = dev_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (m->kind == HS_IDS_U16) {
      e = cudaMemcpyAsync(c->ids, m->ids, c->N * 2, kind, c->stream);
    } else {
      e = cudaMemcpyAsync(c->B[0], m->ids, c->N, kind, c->stream);
      if (e == cudaSuccess) {
        LaunchScope ls(c, HS_K_OTHER);
        e = hs::launch_ids_u8_to_u16((const uint8_t*)c->B[0], c->ids, c->N, c->stream);
      }
    }
    int* maxid = (int*)c->partials;
    if (e == cudaSuccess) e = cudaMemsetAsync(maxid, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
      LaunchScope ls(c, HS_K_OTHER);
      e = hs::launch_max_id(c->ids, c->N, maxid, c->stream);
    }
    int hmax = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hmax, maxid, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      hs_status st = cuda_fail(nullptr, e, "phase-id upload");
      delete c;
      return st;
    }
    if (hmax >= np) {
      delete c;
      return fail(nullptr, HS_ERR_INVALID_ARG, "phase id >= nphase");
    }
  }
  *out = c;
  return HS_OK;
}

hs_status hs_create(hs_ctx** out, const int grid[3], const hs_material* m_in, const double C0[36],
                    const hs_options* opt, void* workspace, size_t workspace_bytes, void* stream) {
  return create_impl(out, grid, m_in, C0, opt, workspace, workspace_bytes, stream, 0);
}

hs_status hs_solve(hs_ctx* c, const double E[6], double tol, int max_iter, void* eps_out, void* sig_out,
                   double sig_eff[6], int* iters, double* final_err) {
  if (!c || !E || !sig_eff) return fail(c, HS_ERR_INVALID_ARG, "null argument");
  if (c->unbound) return fail(c, HS_ERR_INVALID_ARG, "no material: the last hs_set_material failed");
  if (!(tol >= 0) || max_iter < 1) return fail(c, HS_ERR_INVALID_ARG, "bad tol or max_iter");
  double en = 0;
  for (int i = 0; i < 6; ++i) {
    if (!std::isfinite(E[i])) return fail(c, HS_ERR_INVALID_ARG, "non-finite E");
    en += E[i] * E[i];
  }
  if (en == 0 && !c->has_eigen)
    return fail(c, HS_ERR_INVALID_ARG, "E = 0 without eigenstrain (the error norm would divide by <sigma> = 0)");
  if ((eps_out == nullptr) != (sig_out == nullptr)) return fail(c, HS_ERR_INVALID_ARG, "give both or neither field output");
  if (eps_out) {
    cudaPointerAttributes a1, a2;
    cudaError_t e1 = cudaPointerGetAttributes(&a1, eps_out), e2 = cudaPointerGetAttributes(&a2, sig_out);
    if (e1 != cudaSuccess || e2 != cudaSuccess) cudaGetLastError();
    if (e1 != cudaSuccess || e2 != cudaSuccess || (a1.type != cudaMemoryTypeDevice && a1.type != cudaMemoryTypeManaged) ||
        (a2.type != cudaMemoryTypeDevice && a2.type != cudaMemoryTypeManaged))
      return fail(c, HS_ERR_INVALID_ARG, "field outputs must be device pointers");
  }
  c->last_err.clear();
  c->dev_macro = false;
  for (int i = 0; i < 6; ++i) c->Einit[i] = 0;
  if (c->prec == HS_FP32_REFINED)
    return solve_refined(c, E, tol, max_iter, eps_out, sig_out, sig_eff, iters, final_err, nullptr, nullptr, nullptr);
  if (c->f64) return solve_plain<double>(c, E, tol, max_iter, eps_out, sig_out, sig_eff, iters, final_err, nullptr);
  return solve_plain<float>(c, E, tol, max_iter, eps_out, sig_out, sig_eff, iters, final_err, nullptr);
}

hs_status hs_solve_stress(hs_ctx* c, const double S[6], double tol, int max_iter, void* eps_out, void* sig_out,
                          double sig_eff[6], double E_out[6], int* iters, double* final_err) {
  if (!c || !S || !sig_eff) return fail(c, HS_ERR_INVALID_ARG, "null argument");
  if (c->unbound) return fail(c, HS_ERR_INVALID_ARG, "no material: the last hs_set_material failed");
  if (!(tol >= 0) || max_iter < 1) return fail(c, HS_ERR_INVALID_ARG, "bad tol or max_iter");
  double sn = 0;
  for (int i = 0; i < 6; ++i) {
    if (!std::isfinite(S[i])) return fail(c, HS_ERR_INVALID_ARG, "non-finite applied stress");
    sn += S[i] * S[i];
  }
  if (sn == 0 && !c->has_eigen)
    return fail(c, HS_ERR_INVALID_ARG, "applied stress 0 without eigenstrain: the solution is u = 0, E = 0");
  if ((eps_out == nullptr) != (sig_out == nullptr)) return fail(c, HS_ERR_INVALID_ARG, "give both or neither field output");
  if (eps_out) {
    cudaPointerAttributes a1, a2;
    cudaError_t e1 = cudaPointerGetAttributes(&a1, eps_out), e2 = cudaPointerGetAttributes(&a2, sig_out);
    if (e1 != cudaSuccess || e2 != cudaSuccess) cudaGetLastError();
    if (e1 != cudaSuccess || e2 != cudaSuccess || (a1.type != cudaMemoryTypeDevice && a1.type != cudaMemoryTypeManaged) ||
        (a2.type != cudaMemoryTypeDevice && a2.type != cudaMemoryTypeManaged))
      return fail(c, HS_ERR_INVALID_ARG, "field outputs must be device pointers");
  }
  // S0: Voigt stress -> tensor strain components of (lambda0)^-1 : sigma
  double Cinv[36], S0[36];
  if (!inv6(c->C0, Cinv)) return fail(c, HS_ERR_INVALID_ARG, "reference medium is singular");
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) S0[i * 6 + j] = (i < 3 ? 1.0 : 0.5) * Cinv[i * 6 + j];
  // initial guess E = (lambda0)^-1 : sigma^a (Algorithm 1)
  double E0[6];
  for (int i = 0; i < 6; ++i) {
    double acc = 0;
    for (int j = 0; j < 6; ++j) acc += S0[i * 6 + j] * S[j];
    E0[i] = acc;
  }
  c->last_err.clear();
  double Efin[6];
  hs_status st;
  if (c->prec == HS_FP32_REFINED) {
    c->dev_macro = false;
    for (int i = 0; i < 6; ++i) c->Einit[i] = 0;
    st = solve_refined(c, E0, tol, max_iter, eps_out, sig_out, sig_eff, iters, final_err, S, S0, Efin);
  } else {
    double host_macro[42];
    for (int i = 0; i < 6; ++i) host_macro[i] = S[i];
    for (int i = 0; i < 36; ++i) host_macro[6 + i] = S0[i];
    cudaError_t e = cudaMemcpyAsync(c->macro, host_macro, sizeof(host_macro), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "applied stress upload");
    c->dev_macro = true;
    for (int i = 0; i < 6; ++i) c->Einit[i] = E0[i];
    st = c->f64 ? solve_plain<double>(c, E0, tol, max_iter, eps_out, sig_out, sig_eff, iters, final_err, Efin)
                : solve_plain<float>(c, E0, tol, max_iter, eps_out, sig_out, sig_eff, iters, final_err, Efin);
    c->dev_macro = false;
    for (int i = 0; i < 6; ++i) c->Einit[i] = 0;
  }
  if (st >= 0 && E_out)
    for (int i = 0; i < 6; ++i) E_out[i] = Efin[i];
  return st;
}

// captured chunks hold kernel arguments: drop them when an argument changes
static void drop_graphs(hs_ctx* c) {
  for (int i = 0; i < 2; ++i) drop_graph(c, i, true);
}

hs_status hs_set_eigenstrain(hs_ctx* c, const double* eps0) {
  if (!c) return HS_ERR_INVALID_ARG;
  drop_graphs(c);
  if (eps0 == nullptr) {
    c->has_eigen = false;
    return HS_OK;
  }
  std::vector<double> s0d((size_t)c->nphase * 6);
  std::vector<float> s0f((size_t)c->nphase * 6);
  bool any = false;
  for (int p = 0; p < c->nphase; ++p) {
    const double* e = eps0 + (size_t)p * 6;
    double eng[6];
    for (int i = 0; i < 6; ++i) {
      if (!std::isfinite(e[i])) return fail(c, HS_ERR_INVALID_ARG, "non-finite eigenstrain");
      eng[i] = (i < 3 ? 1.0 : 2.0) * e[i];
      any = any || e[i] != 0;
    }
    const double* C = c->table.data() + (size_t)p * 36;
    for (int i = 0; i < 6; ++i) {
      double acc = 0;
      for (int j = 0; j < 6; ++j) acc += C[i * 6 + j] * eng[j];
      s0d[(size_t)p * 6 + i] = acc;
      s0f[(size_t)p * 6 + i] = (float)acc;
    }
  }
  cudaError_t e = cudaMemcpyAsync(c->sig0d, s0d.data(), s0d.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->sig0f, s0f.data(), s0f.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "eigenstrain upload");
  c->has_eigen = any;
  return HS_OK;
}

hs_status hs_create_sized(hs_ctx** out, const int grid[3], const hs_material* m, const double C0[36],
                          const hs_options* opt, int layout_nphase, void* workspace, size_t workspace_bytes,
                          void* stream) {
  if (layout_nphase < 1 || layout_nphase > HS_MAX_PHASES)
    return fail(nullptr, HS_ERR_INVALID_ARG, "layout_nphase out of range");
  return create_impl(out, grid, m, C0, opt, workspace, workspace_bytes, stream, layout_nphase);
}

hs_status hs_set_material(hs_ctx* c, const hs_material* m, const double C0[36]) {
  if (!c || !m) return fail(c, HS_ERR_INVALID_ARG, "null argument");
  if (m->kind != HS_COEFFS_F32 && m->nphase > c->layout_np)
    return fail(c, HS_ERR_INVALID_ARG, "more phases than the workspace was sized for");
  const int grid[3] = {c->n1, c->n2, c->n3};
  // a fresh context on the same workspace, with the same options and layout, uploads the
  // material and chooses the reference medium; this context takes its material state
  hs_ctx* t = nullptr;
  c->unbound = true;
  hs_status s = create_impl(&t, grid, m, C0, &c->opt, c->ws, c->ws_bytes, c->stream, c->layout_np);
  if (s != HS_OK) return fail(c, s, std::string("hs_set_material: ") + g_last_error);
  if (t->layout_np != c->layout_np) {
    hs_destroy(t);
    return fail(c, HS_ERR_INVALID_ARG, "more phases than the workspace was sized for");
  }
  // captured graphs hold the constitutive-law variant, a general reference medium's
  // coefficients and the eigenstrain pointer as kernel arguments
  const bool same_kernels = (t->iso == c->iso) && t->c0_iso && c->c0_iso && !c->has_eigen;
  if (!same_kernels) drop_graphs(c);
  c->nphase = t->nphase;
  c->iso = t->iso;
  c->table = t->table;
  memcpy(c->C0, t->C0, sizeof(c->C0));
  memcpy(c->G6, t->G6, sizeof(c->G6));
  c->c0_iso = t->c0_iso;
  c->c0_a = t->c0_a;
  c->c0_b = t->c0_b;
  c->has_eigen = false;
  c->warm = false;
  c->unbound = false;
  for (int k = 0; k < HS_K_COUNT; ++k) c->launches[k] += t->launches[k];
  hs_destroy(t);
  return HS_OK;
}

hs_status hs_get_displacement(hs_ctx* c, double* u) {
  if (!c || !u) return fail(c, HS_ERR_INVALID_ARG, "null argument");
  cudaError_t e;
  const size_t n = 3 * c->N;
  if (c->prec == HS_FP32_REFINED) {
    e = cudaMemcpyAsync(u, c->u64, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  } else if (c->f64) {
    e = cudaMemcpyAsync(u, c->B[1], n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  } else {
    e = hs::launch_f32_to_f64((const float*)c->B[1], u, n, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "displacement export");
  return HS_OK;
}

hs_status hs_err_history(const hs_ctx* c, double* out, int n, int* n_written) {
  if (!c || (!out && n > 0) || n < 0) return HS_ERR_INVALID_ARG;
  const int k = std::min(n, (int)c->hist_host.size());
  for (int i = 0; i < k; ++i) out[i] = c->hist_host[i];
  if (n_written) *n_written = k;
  return HS_OK;
}

hs_status hs_get_state(hs_ctx* c, void* uhat) {
  if (!c || !uhat) return fail(c, HS_ERR_INVALID_ARG, "null argument");
  if (c->prec == HS_FP32_REFINED) return fail(c, HS_ERR_INVALID_ARG, "state export is not available in refined mode");
  cudaError_t e = c->f64 ? hs::launch_state_export<double>((const double2*)c->S, (double2*)uhat, c->n2, c->n3, c->nh, c->P, c->stream)
                         : hs::launch_state_export<float>((const float2*)c->S, (double2*)uhat, c->n2, c->n3, c->nh, c->P, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "state export");
  return HS_OK;
}

hs_status hs_set_state(hs_ctx* c, const void* uhat) {
  if (!c || !uhat) return fail(c, HS_ERR_INVALID_ARG, "null argument");
  if (c->prec == HS_FP32_REFINED) return fail(c, HS_ERR_INVALID_ARG, "state import is not available in refined mode");
  cudaError_t e = c->f64 ? hs::launch_state_import<double>((const double2*)uhat, (double2*)c->S, c->n2, c->n3, c->nh, c->P, c->stream)
                         : hs::launch_state_import<float>((const double2*)uhat, (float2*)c->S, c->n2, c->n3, c->nh, c->P, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "state import");
  c->warm = true;
  return HS_OK;
}

// --------------------------------------------------------------------------
// Autotuner: time candidate tilings on the caller's workspace and keep the
// fastest per (grid, precision, isotropy) in a process-wide plan cache.
// --------------------------------------------------------------------------
namespace {
struct PlanKey {
  int n1, n2, n3, prec, iso;
  bool operator<(const PlanKey& o) const {
    return std::tie(n1, n2, n3, prec, iso) < std::tie(o.n1, o.n2, o.n3, o.prec, o.iso);
  }
};
std::mutex g_plan_mu;
std::map<PlanKey, hs_options> g_plans;

bool table_isotropic(const double* table, int nphase) {
  for (int p = 0; p < nphase; ++p) {
    const double* C = table + (size_t)p * 36;
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
  }
  return true;
}
}  // namespace

hs_status hs_autotune(const int grid[3], const hs_material* m_in, const hs_options* base, void* workspace,
                      size_t workspace_bytes, void* stream, int iters, hs_options* best, double* best_ms) {
  if (!grid || !m_in || !best || iters < 1) return fail(nullptr, HS_ERR_INVALID_ARG, "bad argument");
  IdsMaterial im;
  if (m_in->kind == HS_COEFFS_F32 && check_grid(grid) != HS_OK)
    return fail(nullptr, HS_ERR_UNSUPPORTED_SIZE, "unsupported grid size");
  {
    hs_status sm = to_ids_material(m_in, grid, stream, &im);
    if (sm != HS_OK) return fail(nullptr, sm, sm == HS_ERR_CUDA ? g_last_error : "bad per-voxel stiffness field");
  }
  const hs_material* m = im.use;
  if (!m->table) return fail(nullptr, HS_ERR_INVALID_ARG, "bad argument");
  hs_options b;
  hs_default_options(&b);
  if (base) b = *base;
  const PlanKey key{grid[0], grid[1], grid[2], b.precision, table_isotropic(m->table, m->nphase) ? 1 : 0};
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
      *best = it->second;
      if (best_ms) *best_ms = -1.0;  // from the cache, not re-timed
      return HS_OK;
    }
  }
  // candidates: y tile x z chunk of the real-space pass (blocks targeted at 512 .. 4096), then
  // the column tile width and the z pass's state staging
  std::vector<hs_options> cands;
  for (int ty : {2, 4, 8}) {
    if (grid[1] % ty != 0) continue;
    std::vector<int> zcs;
    const int ytiles = grid[1] / ty;
    for (int target : {512, 1024, 2048, 4096}) {
      const int nz = std::max(1, std::min(grid[2], (target + ytiles - 1) / ytiles));
      const int zc = (grid[2] + nz - 1) / nz;
      if (std::find(zcs.begin(), zcs.end(), zc) == zcs.end()) zcs.push_back(zc);
    }
    for (int zc : zcs) {
      hs_options o = b;
      o.ytile = ty;
      o.zchunk = zc;
      cands.push_back(o);
    }
  }
  const double E[6] = {1e-3, 0, 0, 0, 0, 0};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(nullptr, HS_ERR_CUDA, "event create");
  auto time_one = [&](const hs_options& o, double* ms) -> hs_status {
    hs_ctx* c = nullptr;
    hs_status st = hs_create(&c, grid, m, nullptr, &o, workspace, workspace_bytes, stream);
    if (st != HS_OK) return st;
    double se[6];
    int it = 0;
    double err = 0;
    st = hs_solve(c, E, 0.0, iters, nullptr, nullptr, se, &it, &err);  // warm-up (and graph capture)
    if (st >= 0) {
      cudaEventRecord(e0, s);
      st = hs_solve(c, E, 0.0, iters, nullptr, nullptr, se, &it, &err);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      *ms = t / std::max(1, it);
    }
    hs_destroy(c);
    return st < 0 ? st : HS_OK;
  };
  double best_t = 1e300;
  hs_options win = b;
  for (const hs_options& o : cands) {
    double t = 0;
    if (time_one(o, &t) == HS_OK && t < best_t) {
      best_t = t;
      win = o;
    }
  }
  {
    hs_options o = win;  // the wider column tile
    o.col_tile = (b.precision == HS_FP64) ? 8 : 16;
    double t = 0;
    if (time_one(o, &t) == HS_OK && t < best_t) {
      best_t = t;
      win = o;
    }
  }
  for (int cs : {1, 2}) {
    hs_options o = win;  // the z pass's state staging
    o.col_state = cs;
    double t = 0;
    if (time_one(o, &t) == HS_OK && t < best_t) {
      best_t = t;
      win = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!(best_t < 1e300)) return fail(nullptr, HS_ERR_CUDA, "no candidate ran");
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    g_plans[key] = win;
  }
  *best = win;
  if (best_ms) *best_ms = best_t;
  return HS_OK;
}

hs_status hs_get_reference_medium(const hs_ctx* c, double C0[36]) {
  if (!c || !C0) return HS_ERR_INVALID_ARG;
  memcpy(C0, c->C0, sizeof(c->C0));
  return HS_OK;
}

hs_status hs_profile_enable(hs_ctx* c, int on) {
  if (!c || on < 0) return HS_ERR_INVALID_ARG;
  c->prof = (on != 0);
  c->prof_every = on > 0 ? on : 1;
  c->chunk_seq = 0;
  return HS_OK;
}

hs_status hs_profile_read(hs_ctx* c, double ms[HS_K_COUNT], long long launches[HS_K_COUNT]) {
  if (!c || !ms || !launches) return HS_ERR_INVALID_ARG;
  for (int k = 0; k < HS_K_COUNT; ++k) ms[k] = 0;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile read");
  for (auto& ev : c->ev_used) {
    float t = 0;
    if (cudaEventElapsedTime(&t, ev.a, ev.b) == cudaSuccess) ms[ev.kind] += t;
    c->ev_pool.push_back(ev.a);
    c->ev_pool.push_back(ev.b);
  }
  c->ev_used.clear();
  for (int k = 0; k < HS_K_COUNT; ++k) {
    // sampled profiling: the timed launches' total, scaled to all launches of the class
    if (c->timed[k] > 0 && c->timed[k] < c->launches[k]) ms[k] *= (double)c->launches[k] / (double)c->timed[k];
    launches[k] = c->launches[k];
    c->launches[k] = 0;
    c->timed[k] = 0;
  }
  return HS_OK;
}

hs_status hs_compress_coefficients(const int grid[3], const float* coeffs, unsigned short* ids, double* table,
                                   int capacity, int* nphase) {
  if (!grid || !coeffs || !ids || !table || !nphase || capacity < 1)
    return fail(nullptr, HS_ERR_INVALID_ARG, "null argument or capacity < 1");
  for (int i = 0; i < 3; ++i)
    if (grid[i] < 1) return fail(nullptr, HS_ERR_INVALID_ARG, "grid entry < 1");
  const size_t N = (size_t)grid[0] * grid[1] * grid[2];
  CoeffCompressor cc(N, capacity);
  const float* comp[21];
  for (int c = 0; c < 21; ++c) comp[c] = coeffs + (size_t)c * N;
  hs_status s = cc.add(comp, N, 0);
  if (s == HS_ERR_UNSUPPORTED_SIZE) return fail(nullptr, s, "more distinct stiffnesses than capacity");
  if (s != HS_OK) return fail(nullptr, s, "non-finite coefficient");
  memcpy(ids, cc.ids.data(), N * sizeof(uint16_t));
  memcpy(table, cc.table.data(), cc.table.size() * sizeof(double));
  *nphase = cc.nphase();
  return HS_OK;
}

void hs_destroy(hs_ctx* c) {
  if (!c) return;
  for (auto& ev : c->ev_used) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  for (int i = 0; i < 2; ++i) drop_graph(c, i, true);  // returns the graphs' events to the pool
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

const char* hs_error_string(hs_status s) {
  switch (s) {
    case HS_OK: return "converged";
    case HS_NOT_CONVERGED: return "max_iter reached before err < tol";
    case HS_ERR_INVALID_ARG: return "invalid argument";
    case HS_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
    case HS_ERR_OOM: return "workspace too small";
    case HS_ERR_CUDA: return "CUDA error";
    case HS_DIVERGED: return "iteration diverged";
    case HS_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* hs_last_error(const hs_ctx* c) {
  if (c) return c->last_err.c_str();
  return g_last_error.c_str();
}


// --------------------------------------------------------------------------
// Batched solves: many RVEs and load cases in shared launches.  Items (an RVE
// under one macroscopic strain) of the same grid and phase isotropy form a size
// class; each item has a full single-solve workspace, the items of a class lie
// one stride apart, and every kernel of the class runs as one launch over all
// its items (grid.z = item).  A chunk of iterations of every class is captured
// as one CUDA graph, the classes on forked streams, and replayed until every
// item has stopped.  Each item keeps its own device status, so an item that
// converges stops on its own while the others go on.
// --------------------------------------------------------------------------
}  // extern "C"

struct hs_batch {
  struct Class {
    int n1, n2, n3;
    bool iso;
    int max_np;
    size_t stride;
    std::vector<int> items;      // item indices in this class, in workspace order
    std::vector<hs_ctx*> ctx;    // one context per item (ctx[0] drives the batched launches)
    cudaStream_t s = nullptr;
    cudaEvent_t joined = nullptr;
    std::vector<DevStatus> hst;  // host copies of the items' statuses
  };
  std::vector<Class> cls;
  std::vector<int> item_cls, item_pos;
  int nitem = 0;
  hs_options opt;
  bool f64 = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int gchunks[2] = {0, 0};
  std::vector<std::vector<double>> hist;  // per item: errors (refined: FP64 sweeps; else every evaluation)
  std::string last_err;
};

namespace {

hs_status bfail(hs_batch* b, hs_status s, const std::string& msg) {
  g_last_error = msg;
  if (b) b->last_err = msg;
  return s;
}

struct ClassKey {
  int n1, n2, n3, iso;
  bool operator<(const ClassKey& o) const {
    return std::tie(n1, n2, n3, iso) < std::tie(o.n1, o.n2, o.n3, o.iso);
  }
};

// Size classes of a batch, in order of first appearance; stride and bytes per class.
hs_status batch_classes(int nrve, const int* grids, const hs_material* mats, const int* nphase, int nitem,
                        const int* item_rve, int prec, std::vector<hs_batch::Class>* out,
                        std::vector<int>* item_cls, std::vector<int>* item_pos, size_t* total) {
  if (nrve < 1 || nitem < 1 || !grids || !item_rve) return HS_ERR_INVALID_ARG;
  std::map<ClassKey, int> index;
  std::vector<int> rve_iso(nrve);
  for (int r = 0; r < nrve; ++r) {
    hs_status s = check_grid(grids + 3 * r);
    if (s != HS_OK) return s;
    const int np = mats ? mats[r].nphase : nphase[r];
    if (np < 1 || np > HS_MAX_PHASES) return HS_ERR_INVALID_ARG;
    if (mats) {
      if ((mats[r].kind != HS_IDS_U8 && mats[r].kind != HS_IDS_U16) || !mats[r].ids || !mats[r].table)
        return HS_ERR_INVALID_ARG;
      rve_iso[r] = table_isotropic(mats[r].table, np) ? 1 : 0;
    } else {
      rve_iso[r] = 0;  // sizing only: isotropy does not change the layout
    }
  }
  out->clear();
  item_cls->assign(nitem, 0);
  item_pos->assign(nitem, 0);
  for (int i = 0; i < nitem; ++i) {
    const int r = item_rve[i];
    if (r < 0 || r >= nrve) return HS_ERR_INVALID_ARG;
    const int* g = grids + 3 * r;
    const ClassKey k{g[0], g[1], g[2], rve_iso[r]};
    auto it = index.find(k);
    int ci;
    if (it == index.end()) {
      ci = (int)out->size();
      index.emplace(k, ci);
      hs_batch::Class c;
      c.n1 = g[0];
      c.n2 = g[1];
      c.n3 = g[2];
      c.iso = rve_iso[r] != 0;
      c.max_np = 0;
      c.stride = 0;
      out->push_back(c);
    } else {
      ci = it->second;
    }
    hs_batch::Class& c = (*out)[ci];
    (*item_cls)[i] = ci;
    (*item_pos)[i] = (int)c.items.size();
    c.items.push_back(i);
    c.max_np = std::max(c.max_np, mats ? mats[r].nphase : nphase[r]);
  }
  size_t off = 0;
  for (auto& c : *out) {
    c.stride = align256(make_layout(c.n1, c.n2, c.n3, c.max_np, prec).total);
    off += c.stride * c.items.size();
  }
  *total = off;
  return HS_OK;
}

// status records of every item of class c: host copies -> device (reset) or device -> host (read)
hs_status batch_put_status(hs_batch* b, hs_batch::Class& c) {
  hs_ctx* L = c.ctx[0];
  cudaError_t e = cudaMemcpy2DAsync(L->st, c.stride, c.hst.data(), sizeof(DevStatus), sizeof(DevStatus), c.items.size(),
                                    cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("status upload: ") + cudaGetErrorString(e));
  return HS_OK;
}

hs_status batch_get_status(hs_batch* b) {
  for (auto& c : b->cls) {
    hs_ctx* L = c.ctx[0];
    cudaError_t e = cudaMemcpy2DAsync(c.hst.data(), sizeof(DevStatus), L->st, c.stride, sizeof(DevStatus),
                                      c.items.size(), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
  return HS_OK;
}

void status_init(DevStatus* h, const hs_ctx* c, double tol, int max_iter, double denom, const double* E, double rel_tol,
                 bool retired) {
  memset(h, 0, sizeof(*h));
  h->max_iter = max_iter;
  h->hist_cap = kHistCap;
  h->tol = tol;
  h->denom = denom;
  h->nvox = (double)c->N;
  h->rel_tol = rel_tol;
  h->retired = retired ? 1 : 0;
  h->done = retired ? hs::DONE_CONVERGED : hs::DONE_RUNNING;
  for (int i = 0; i < 6; ++i) h->E[i] = E ? E[i] : 0.0;
}

hs_status batch_zero_state(hs_batch* b) {
  for (auto& c : b->cls)
    for (hs_ctx* x : c.ctx) {
      cudaError_t e = cudaMemsetAsync(x->S, 0, cbuf_bytes(x), b->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(x->B[0], 0, cbuf_bytes(x), b->stream);
      if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("state reset: ") + cudaGetErrorString(e));
    }
  return HS_OK;
}

// Run fn(lead) for every class on the class's stream, forked from and joined to
// the batch stream (so classes overlap on the device).
template <typename F> hs_status batch_fork(hs_batch* b, F fn) {
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("fork: ") + cudaGetErrorString(e));
  for (auto& c : b->cls) {
    hs_ctx* L = c.ctx[0];
    e = cudaStreamWaitEvent(c.s, b->fork, 0);
    if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("fork: ") + cudaGetErrorString(e));
    cudaStream_t keep = L->stream;
    L->stream = c.s;
    hs_status st = fn(L);
    L->stream = keep;
    if (st != HS_OK) return bfail(b, st, L->last_err);
    e = cudaEventRecord(c.joined, c.s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, c.joined, 0);
    if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("join: ") + cudaGetErrorString(e));
  }
  return HS_OK;
}

void batch_drop_graph(hs_batch* b, int gi) {
  if (b->gexec[gi]) cudaGraphExecDestroy(b->gexec[gi]);
  b->gexec[gi] = nullptr;
  for (auto& c : b->cls) drop_graph(c.ctx[0], gi, false);
}

// Basic-scheme iterations of every item until every item's status says done.
template <typename T> hs_status batch_iterate(hs_batch* b, bool with_src) {
  const int gi = with_src ? 1 : 0;
  const int chunk = std::max(1, b->opt.check_every);
  const double zeroE[6] = {0, 0, 0, 0, 0, 0};
  auto one_chunk = [&](hs_ctx* L) -> hs_status {
    for (int i = 0; i < chunk; ++i) {
      hs_status s = launch_rows<T>(L, hs::ROW_C2R, nullptr, true);
      if (s == HS_OK) s = launch_stencil<T>(L, zeroE, with_src ? L->rsrc : nullptr, hs::MODE_FORCE, nullptr, nullptr);
      if (s == HS_OK) s = launch_rows<T>(L, hs::ROW_R2C, nullptr, true);
      if (s == HS_OK) s = launch_cols<T>(L, 0);
      if (s != HS_OK) return s;
    }
    return HS_OK;
  };
  const bool graphs = b->opt.use_graphs && b->stream != nullptr && b->stream != cudaStreamLegacy &&
                      b->stream != cudaStreamPerThread;
  for (;;) {
    if (graphs && b->gexec[gi] != nullptr) {
      cudaError_t e = cudaGraphLaunch(b->gexec[gi], b->stream);
      if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
      for (auto& c : b->cls) account_replay(c.ctx[0], gi);
    } else if (graphs && b->gchunks[gi] >= 1) {
      batch_drop_graph(b, gi);
      cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
      for (auto& c : b->cls) {
        c.ctx[0]->capturing = true;
        c.ctx[0]->cap_gi = gi;
      }
      hs_status s = batch_fork(b, one_chunk);
      for (auto& c : b->cls) c.ctx[0]->capturing = false;
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(b->stream, &g);
      cudaGraphExec_t ex = nullptr;
      if (s == HS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
      if (g) cudaGraphDestroy(g);
      if (s != HS_OK || e != cudaSuccess) {
        cudaGetLastError();
        batch_drop_graph(b, gi);
        return s != HS_OK ? s : bfail(b, HS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      }
      b->gexec[gi] = ex;
      e = cudaGraphLaunch(ex, b->stream);
      if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
      for (auto& c : b->cls) account_replay(c.ctx[0], gi);
    } else {
      hs_status s = batch_fork(b, one_chunk);
      if (s != HS_OK) return s;
      ++b->gchunks[gi];
    }
    hs_status s = batch_get_status(b);
    if (s != HS_OK) return s;
    bool all = true;
    for (auto& c : b->cls)
      for (auto& h : c.hst)
        if (!h.retired && !h.done) all = false;
    if (all) return HS_OK;
  }
}

// u64 += inverse transform of every item's correction state (refined mode)
hs_status batch_accumulate(hs_batch* b) {
  return batch_fork(b, [&](hs_ctx* L) -> hs_status {
    hs_status s = launch_state_to_buf<float>(L, 0);
    if (s == HS_OK) s = launch_rows<float>(L, hs::ROW_C2R, L->u64, false);
    return s;
  });
}

}  // namespace

extern "C" {

hs_status hs_batch_workspace_size(int nrve, const int* grids, const int* nphase, int nitem, const int* item_rve,
                                  const hs_options* opt, size_t* bytes) {
  if (!grids || !nphase || !item_rve || !bytes) return fail(nullptr, HS_ERR_INVALID_ARG, "null argument");
  hs_options o;
  hs_default_options(&o);
  if (opt) o = *opt;
  if (o.precision < HS_FP64 || o.precision > HS_FP32_REFINED) return fail(nullptr, HS_ERR_INVALID_ARG, "bad precision");
  std::vector<hs_batch::Class> cls;
  std::vector<int> ic, ip;
  size_t total = 0;
  hs_status s = batch_classes(nrve, grids, nullptr, nphase, nitem, item_rve, o.precision, &cls, &ic, &ip, &total);
  if (s != HS_OK) return fail(nullptr, s, "bad batch description");
  *bytes = total;
  return HS_OK;
}

hs_status hs_batch_create(hs_batch** out, int nrve, const int* grids, const hs_material* mats, int nitem,
                          const int* item_rve, const hs_options* opt, int autotune, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (!out || !grids || !mats || !item_rve || !workspace) return fail(nullptr, HS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return fail(nullptr, HS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  hs_options o;
  hs_default_options(&o);
  if (opt) o = *opt;
  if (o.xfuse != 0) return fail(nullptr, HS_ERR_INVALID_ARG, "batched solves run the split x-pass (xfuse = 0)");
  if (o.precision < HS_FP64 || o.precision > HS_FP32_REFINED) return fail(nullptr, HS_ERR_INVALID_ARG, "bad precision");
  hs_batch* b = new hs_batch();
  size_t total = 0;
  hs_status s = batch_classes(nrve, grids, mats, nullptr, nitem, item_rve, o.precision, &b->cls, &b->item_cls,
                              &b->item_pos, &total);
  if (s != HS_OK) {
    delete b;
    return fail(nullptr, s, "bad batch description (grid, material kind, phase count or item index)");
  }
  if (workspace_bytes < total) {
    delete b;
    return fail(nullptr, HS_ERR_OOM, "workspace too small for the batch");
  }
  b->nitem = nitem;
  b->opt = o;
  b->f64 = (o.precision == HS_FP64);
  b->stream = static_cast<cudaStream_t>(stream);
  b->hist.assign(nitem, {});
  auto undo = [&](hs_status st, const std::string& msg) {
    hs_batch_destroy(b);
    return fail(nullptr, st, msg);
  };
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return undo(HS_ERR_CUDA, "event create");
  char* base = static_cast<char*>(workspace);
  for (auto& c : b->cls) {
    if (cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.joined, cudaEventDisableTiming) != cudaSuccess)
      return undo(HS_ERR_CUDA, "stream create");
    hs_options oc = o;
    const int grid[3] = {c.n1, c.n2, c.n3};
    if (autotune) {
      // the class's tiling from the plan cache (tuned on the class's first workspace on a miss)
      hs_options best;
      const hs_material& m0 = mats[item_rve[c.items[0]]];
      if (hs_autotune(grid, &m0, &o, base, c.stride, stream, 8, &best, nullptr) == HS_OK) oc = best;
    }
    for (size_t k = 0; k < c.items.size(); ++k) {
      hs_ctx* x = nullptr;
      const int r = item_rve[c.items[k]];
      s = create_impl(&x, grid, &mats[r], nullptr, &oc, base + k * c.stride, c.stride, stream, c.max_np);
      if (s != HS_OK) return undo(s, std::string("item ") + std::to_string(c.items[k]) + ": " + g_last_error);
      if (x->iso != c.iso || !x->c0_iso) {
        hs_destroy(x);
        return undo(HS_ERR_INVALID_ARG, "batched items need an isotropic reference medium");
      }
      c.ctx.push_back(x);
    }
    c.ctx[0]->batch_n = (int)c.items.size();
    c.ctx[0]->batch_stride = c.stride;
    c.hst.resize(c.items.size());
    base += c.stride * c.items.size();
  }
  *out = b;
  return HS_OK;
}

hs_status hs_batch_solve(hs_batch* b, const double* E, double tol, int max_iter, double* sig_eff, int* iters,
                         double* final_err, int* status) {
  if (!b || !E || !sig_eff || !iters || !final_err || !status) return bfail(b, HS_ERR_INVALID_ARG, "null argument");
  if (!(tol >= 0) || max_iter < 1) return bfail(b, HS_ERR_INVALID_ARG, "bad tol or max_iter");
  for (int i = 0; i < b->nitem; ++i) {
    double en = 0;
    for (int k = 0; k < 6; ++k) {
      if (!std::isfinite(E[6 * i + k])) return bfail(b, HS_ERR_INVALID_ARG, "non-finite E");
      en += E[6 * i + k] * E[6 * i + k];
    }
    if (en == 0) return bfail(b, HS_ERR_INVALID_ARG, "E = 0 (the error norm would divide by <sigma> = 0)");
  }
  b->last_err.clear();
  for (auto& h : b->hist) h.clear();
  const int n = b->nitem;
  std::vector<int> total(n, 0), done(n, 0);
  std::vector<hs_status> st(n, HS_NOT_CONVERGED);
  auto item_status = [&](int i) -> DevStatus& { return b->cls[b->item_cls[i]].hst[b->item_pos[i]]; };
  auto item_ctx = [&](int i) -> hs_ctx* { return b->cls[b->item_cls[i]].ctx[b->item_pos[i]]; };
  auto finish = [&](int i, const DevStatus& h, hs_status s) {
    for (int k = 0; k < 6; ++k) sig_eff[6 * i + k] = h.sig_mean[k];
    final_err[i] = h.err;
    st[i] = s;
    done[i] = 1;
  };
  hs_status s;
  if (b->opt.precision != HS_FP32_REFINED) {
    for (int i = 0; i < n; ++i) status_init(&item_status(i), item_ctx(i), tol, max_iter, 0.0, E + 6 * i, 0.0, false);
    for (auto& c : b->cls)
      if ((s = batch_put_status(b, c)) != HS_OK) return s;
    if ((s = batch_zero_state(b)) != HS_OK) return s;
    s = b->f64 ? batch_iterate<double>(b, false) : batch_iterate<float>(b, false);
    if (s != HS_OK) return s;
    for (int i = 0; i < n; ++i) {
      const DevStatus& h = item_status(i);
      total[i] = h.evals;
      finish(i, h, status_code(h));
      hs_ctx* x = item_ctx(i);
      const int k = std::min(h.evals, kHistCap);
      b->hist[i].resize(k);
      if (k) {
        cudaError_t e = cudaMemcpyAsync(b->hist[i].data(), x->hist, k * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, "history read");
      }
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, "history read");
  } else {
    // FP32 iterations with FP64 residual sweeps, every item in step: first the plain FP32
    // solve from u = 0 (the correction equation of u = 0 is the problem itself), then
    // alternately an FP64 sweep (which takes every stop decision) and an FP32 correction solve.
    const double zeroE[6] = {0, 0, 0, 0, 0, 0};
    for (auto& c : b->cls)
      for (hs_ctx* x : c.ctx) {
        cudaError_t e = cudaMemsetAsync(x->u64, 0, 3 * x->N * sizeof(double), b->stream);
        if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, "u64 reset");
      }
    if (max_iter > 1) {
      const int budget = std::min(std::max(1, b->opt.inner_max), max_iter - 1);
      for (int i = 0; i < n; ++i)
        status_init(&item_status(i), item_ctx(i), 0.0, budget, 0.0, E + 6 * i, b->opt.inner_ratio, false);
      for (auto& c : b->cls)
        if ((s = batch_put_status(b, c)) != HS_OK) return s;
      if ((s = batch_zero_state(b)) != HS_OK) return s;
      if ((s = batch_iterate<float>(b, false)) != HS_OK) return s;
      for (int i = 0; i < n; ++i) {
        const DevStatus& h = item_status(i);
        total[i] += h.evals;
        if (h.done == hs::DONE_DIVERGED) finish(i, h, HS_DIVERGED);
      }
      for (int i = 0; i < n; ++i) item_status(i).retired = done[i];
      for (auto& c : b->cls)
        if ((s = batch_put_status(b, c)) != HS_OK) return s;
      if ((s = batch_accumulate(b)) != HS_OK) return s;
    }
    for (;;) {
      for (int i = 0; i < n; ++i)
        status_init(&item_status(i), item_ctx(i), 0.0, 1 << 30, 0.0, E + 6 * i, 0.0, done[i] != 0);
      for (auto& c : b->cls)
        if ((s = batch_put_status(b, c)) != HS_OK) return s;
      s = batch_fork(b, [&](hs_ctx* L) { return launch_residual64(L, zeroE, hs::MODE_FORCE, nullptr, nullptr); });
      if (s != HS_OK) return s;
      if ((s = batch_get_status(b)) != HS_OK) return s;
      bool any = false;
      for (int i = 0; i < n; ++i) {
        if (done[i]) continue;
        const DevStatus& h = item_status(i);
        total[i] += 1;
        b->hist[i].push_back(h.err);
        if (!(h.err == h.err) || h.err > 1e300) finish(i, h, HS_DIVERGED);
        else if (h.err < tol) finish(i, h, HS_OK);
        else if (total[i] >= max_iter) finish(i, h, HS_NOT_CONVERGED);
        else any = true;
      }
      if (!any) break;
      // correction solves K du = -r in FP32 (source r, macro strain 0) for the items still running
      std::vector<double> err64(n), norm64(n);
      for (int i = 0; i < n; ++i) {
        err64[i] = item_status(i).err;
        norm64[i] = item_status(i).sig_norm;
      }
      for (int i = 0; i < n; ++i) {
        const int budget = std::min(std::max(1, b->opt.inner_max), std::max(1, max_iter - total[i]));
        status_init(&item_status(i), item_ctx(i), b->opt.inner_ratio * err64[i], budget, norm64[i], zeroE, 0.0,
                    done[i] != 0);
      }
      for (auto& c : b->cls)
        if ((s = batch_put_status(b, c)) != HS_OK) return s;
      if ((s = batch_zero_state(b)) != HS_OK) return s;
      if ((s = batch_iterate<float>(b, true)) != HS_OK) return s;
      for (int i = 0; i < n; ++i) {
        if (done[i]) continue;
        const DevStatus& h = item_status(i);
        total[i] += h.evals;
        if (h.done == hs::DONE_DIVERGED) finish(i, h, HS_DIVERGED);
      }
      for (int i = 0; i < n; ++i) item_status(i).retired = done[i];
      for (auto& c : b->cls)
        if ((s = batch_put_status(b, c)) != HS_OK) return s;
      if ((s = batch_accumulate(b)) != HS_OK) return s;
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, HS_ERR_CUDA, "batch sync");
  }
  bool all_ok = true;
  for (int i = 0; i < n; ++i) {
    iters[i] = total[i];
    status[i] = st[i];
    if (st[i] != HS_OK) all_ok = false;
  }
  return all_ok ? HS_OK : HS_NOT_CONVERGED;
}

hs_status hs_batch_err_history(const hs_batch* b, int item, double* out, int n, int* n_written) {
  if (!b || item < 0 || item >= b->nitem || (!out && n > 0) || n < 0) return HS_ERR_INVALID_ARG;
  const auto& h = b->hist[item];
  const int k = std::min(n, (int)h.size());
  for (int i = 0; i < k; ++i) out[i] = h[i];
  if (n_written) *n_written = k;
  return HS_OK;
}

hs_status hs_batch_launches(hs_batch* b, long long* launches) {
  if (!b || !launches) return HS_ERR_INVALID_ARG;
  long long n = 0;
  for (auto& c : b->cls)
    for (hs_ctx* x : c.ctx)
      for (int k = 0; k < HS_K_COUNT; ++k) {
        n += x->launches[k];
        x->launches[k] = 0;
      }
  *launches = n;
  return HS_OK;
}

hs_status hs_batch_classes(const hs_batch* b, int* nclass, int* class_of_item) {
  if (!b || !nclass) return HS_ERR_INVALID_ARG;
  *nclass = (int)b->cls.size();
  if (class_of_item)
    for (int i = 0; i < b->nitem; ++i) class_of_item[i] = b->item_cls[i];
  return HS_OK;
}

const char* hs_batch_last_error(const hs_batch* b) { return b ? b->last_err.c_str() : g_last_error.c_str(); }

void hs_batch_destroy(hs_batch* b) {
  if (!b) return;
  for (int gi = 0; gi < 2; ++gi)
    if (b->gexec[gi]) cudaGraphExecDestroy(b->gexec[gi]);
  for (auto& c : b->cls) {
    for (hs_ctx* x : c.ctx) hs_destroy(x);
    if (c.s) cudaStreamDestroy(c.s);
    if (c.joined) cudaEventDestroy(c.joined);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

}  // extern "C"
