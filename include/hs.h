/*
 * hs.h -- C ABI of the tetrahedral-stencil FFT homogenization solver for
 * GB300 (sm_103a).
 *
 * The solver computes the discrete mechanical equilibrium of a periodic 3D
 * voxel microstructure under an applied macroscopic strain, with the
 * tetrahedral stencil of Finel, "A fast and robust discrete FFT-based solver
 * for computational homogenization" (arXiv 2405.11168), and iterates the
 * displacement-based basic scheme of its Algorithm 1 (Section 2.6):
 *
 *   deps^T1 = D (x)_s u,  deps^T2 = -conj(D) (x)_s u          (Eq. deps_dep_Q)
 *   sigma^T = lambda(r) : (E + deps^T(r))                       (Algorithm 1 step 3)
 *   u(q) <- u(q) - Omega(q).{sigma^T1(q).conj(D) - sigma^T2(q).D}  (Eq. basic_scheme_dep_2)
 *   err  = L2 / ||<sigma>||, stop when err < tol                 (Eqs. L2-norm, tolerance)
 *   eps = E + 1/2 (deps^T1 + deps^T2), sigma = 1/2 (sigma^T1 + sigma^T2)  (Eq. final_fields)
 *
 * Conventions used by every entry point:
 *  - grid[3] = {N1, N2, N3}; real fields are row-major [N3][N2][N1] (x fastest).
 *  - Voigt order 11, 22, 33, 23, 13, 12.  Strains passed in and returned are
 *    TENSOR components (E[3] = eps_23, not gamma_23).  Stiffness matrices are
 *    the engineering 6x6 Voigt matrices (sigma_V = C eps_V with doubled shear
 *    strains), so the tensor components lambda_ijkl equal the Voigt entries.
 *  - Units are the caller's; err is dimensionless.
 *  - Every call runs on the CUDA stream given to hs_create and returns after
 *    the results it reports are on the host.
 *  - Errors are negative hs_status values; on error nothing is written to the
 *    caller's outputs.  No entry point aborts or traps.
 */
#ifndef HS_H
#define HS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hs_ctx hs_ctx; /* opaque, owned by the library */

typedef enum {
  HS_OK = 0,
  HS_NOT_CONVERGED = 1,        /* max_iter reached; outputs hold the last iterate */
  HS_ERR_INVALID_ARG = -1,     /* bad pointer, size, material, tolerance or load */
  HS_ERR_UNSUPPORTED_SIZE = -2,/* N_i odd, < 4, > 512, or with a prime factor other than 2, 3, 5, 7, 11 */
  HS_ERR_OOM = -3,             /* the workspace given is smaller than hs_workspace_size() */
  HS_ERR_CUDA = -4,            /* a CUDA call failed (see hs_last_error) */
  HS_DIVERGED = -5,            /* err became NaN/Inf or grew 1e6x above its minimum */
  HS_ERR_TIMEOUT = -6          /* a bounded device wait (a tensor copy's barrier) gave up */
} hs_status;

enum { HS_FP64 = 0, HS_FP32 = 1, HS_FP32_REFINED = 2 };
enum { HS_IDS_U8 = 0, HS_IDS_U16 = 1, HS_COEFFS_F32 = 2 };
#define HS_MAX_PHASES 65536

/* Microstructure: the stiffness field lambda(r) of Eq. linear_elasticity, either as a phase id per
 * voxel with a stiffness per phase (HS_IDS_U8 / HS_IDS_U16), or as the full 6x6 stiffness of every
 * voxel (HS_COEFFS_F32).  hs_create stores the per-voxel form exactly as phases: voxels whose 21
 * coefficients are identical share a phase (see hs_compress_coefficients), so a field with more
 * than HS_MAX_PHASES distinct stiffnesses is refused with HS_ERR_UNSUPPORTED_SIZE. */
typedef struct {
  int kind;             /* HS_IDS_U8, HS_IDS_U16 or HS_COEFFS_F32 */
  const void* ids;      /* ids kinds: [N3][N2][N1] phase ids; host or device pointer, read during hs_create
                           only.  HS_COEFFS_F32: unused (NULL) */
  const double* table;  /* ids kinds: host pointer, nphase x 36: row-major 6x6 Voigt stiffness per phase;
                           must be symmetric with a non-negative diagonal (C = 0 is a void).
                           HS_COEFFS_F32: unused (NULL) */
  int nphase;           /* ids kinds: 1..HS_MAX_PHASES; every id must be < nphase.  HS_COEFFS_F32: unused */
  const float* coeffs;  /* HS_COEFFS_F32: [21][N3][N2][N1], the upper triangle of each voxel's 6x6 Voigt
                           stiffness in row order (C11 C12 .. C16 C22 .. C26 .. C66), host or device
                           pointer, read during hs_create only; size the workspace with
                           nphase = HS_MAX_PHASES.  Other kinds: unused */
} hs_material;

/* Exact compression of a per-voxel stiffness field (host only; needs no GPU): voxels whose 21
 * coefficients are bit-identical (-0 read as +0) share a phase, numbered in order of first
 * appearance with x fastest.  coeffs: host [21][N3][N2][N1] as hs_material.coeffs; ids: host
 * [N3][N2][N1] output; table: host output, room for `capacity` phases x 36 (symmetric 6x6, the
 * FP32 coefficients widened to FP64); *nphase: phases found.
 * Errors: HS_ERR_INVALID_ARG (null pointer, grid entry < 1, capacity < 1, non-finite coefficient),
 * HS_ERR_UNSUPPORTED_SIZE (more than capacity distinct stiffnesses). */
hs_status hs_compress_coefficients(const int grid[3], const float* coeffs, unsigned short* ids, double* table,
                                   int capacity, int* nphase);

typedef struct {
  int precision;        /* HS_FP64, HS_FP32 or HS_FP32_REFINED */
  int check_every;      /* host polls convergence every this many iterations (>= 1) */
  int out_f32;          /* field outputs as float (1) or double (0) */
  int inner_max;        /* HS_FP32_REFINED: max FP32 iterations per correction solve */
  double inner_ratio;   /* HS_FP32_REFINED: a correction solve stops when its force norm is
                           below inner_ratio times the FP64 residual's; the first solve (from
                           u = 0, the plain FP32 basic scheme) when its error falls to
                           inner_ratio times its first error */
  int zchunk;           /* z planes per block of the x-pass (0 = automatic; a tiling knob that
                           does not change results beyond rounding order) */
  int ytile;            /* y rows per block of the x-pass: 0 = automatic, or 2, 4, 8 dividing N2 */
  int xfuse;            /* 0: x-direction FFTs in their own row passes around a real-space stencil
                           pass (default); 1: one fused x-pass (inverse x FFT, stencil, forward x FFT) */
  int col_tile;         /* y/z FFT tile width in complex columns: 0 = automatic; FP32 8 or 16, FP64 4 or 8
                           (grids with a factor 5, 7 or 11: the automatic width, and xfuse = 0) */
  int col_threads;      /* threads per y/z FFT block: 0 = automatic; a multiple of 32, at most 768 (FP32)
                           or 384 (FP64) */
  int use_graphs;       /* 1 (default): after its first chunk, a solve replays its iteration chunks
                           (check_every iterations) as one captured CUDA graph; 0: plain launches.
                           Chunks that profiling times (hs_profile_enable) run as plain launches. */
  int col_state;        /* z pass + Green update: 0 = automatic, 1 = state read point by point (L2
                           prefetch), 2 = state tile copied to shared memory during the forward z
                           transform (twice the tile's shared memory); results do not change */
  int col_pipe;         /* y passes at lengths 128, 256, 512 with the default tile: 0 = persistent
                           blocks that copy the next tile while transforming the current one
                           (default), 1 = one tile per block, 2 = persistent y passes and a
                           persistent z pass (z lengths 128, 256, 512); results do not change */
  int col_copy;         /* tile loads of the persistent y passes (y lengths 128, 256, 512) and of the
                           z pass (z lengths 64, 128, 256, 512, state read point by point): 0 = tensor
                           (TMA) copies where the driver encodes the tile map, else 16-byte cp.async
                           (default); 1 = cp.async; 2 = as 0, but HS_ERR_UNSUPPORTED_SIZE where such a
                           pass cannot have its map; results do not change.  A tensor copy that does
                           not complete within a bounded wait ends the solve with HS_ERR_TIMEOUT */
} hs_options;

/* Fill *opt with defaults: FP64, check_every 8, double outputs,
 * inner_max 200, inner_ratio 1e-3, zchunk 0, ytile 0, xfuse 0, col_tile 0, col_threads 0,
 * use_graphs 1, col_state 0, col_pipe 0. */
hs_status hs_default_options(hs_options* opt);

/* Autotuner with a process-wide plan cache (no counterpart in the paper: it picks launch
 * shapes, not numerics).  Times `iters` evaluations of each candidate tiling of the
 * real-space and FFT passes (y tile 2/4/8 x z chunk, then the wider column tile and the z
 * pass's col_state) with
 * CUDA events on `stream`, using the caller's workspace (hs_workspace_size bytes for
 * `base`), and writes the fastest options to *best (*best_ms: ms per evaluation, or -1
 * when the plan came from the cache).  Results do not depend on the tiling beyond
 * rounding order.  Keyed by grid, precision and whether all phases are isotropic.
 * Errors: as hs_create / hs_solve; HS_ERR_CUDA if no candidate ran. */
hs_status hs_autotune(const int grid[3], const hs_material* m, const hs_options* base, void* workspace,
                      size_t workspace_bytes, void* stream, int iters, hs_options* best, double* best_ms);

/* Device workspace (bytes) that hs_create needs for this grid, precision and
 * number of phases.  The caller allocates it (e.g. as a PyTorch tensor) and
 * keeps it alive until hs_destroy. */
hs_status hs_workspace_size(const int grid[3], int nphase, const hs_options* opt, size_t* bytes);

/* Create a solver for one microstructure.
 *  grid       N1, N2, N3: even, 4..512, prime factors 2, 3, 5, 7 and 11 only (Section 2.1
 *             requires even N_i).
 *  m          microstructure; copied to the device here.
 *  C0         host 6x6 Voigt stiffness of the homogeneous reference medium lambda0 (Section 2.3),
 *             symmetric positive definite; NULL picks it: for two isotropic phases the rule of the
 *             paper's contrast study (Section 3.4: same Poisson ratio, k0 = a k_m + (1-a) k_i with
 *             a = 0.55 if k_i < k_m else 0.45), otherwise an isotropic medium whose bulk modulus and
 *             shear eigenvalue are the midpoints of the phases' ranges.
 *  opt        options (NULL = defaults).
 *  workspace  device memory of at least hs_workspace_size() bytes, 256-byte aligned, owned by the
 *             caller, in use until hs_destroy.
 *  stream     cudaStream_t to run on (NULL = legacy default stream).
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_UNSUPPORTED_SIZE, HS_ERR_OOM, HS_ERR_CUDA. */
hs_status hs_create(hs_ctx** out, const int grid[3], const hs_material* m, const double C0[36],
                    const hs_options* opt, void* workspace, size_t workspace_bytes, void* stream);

/* hs_create with the workspace layout sized for layout_nphase phases (nphase <= layout_nphase <=
 * HS_MAX_PHASES; size the workspace with hs_workspace_size(grid, layout_nphase, opt)), so that
 * hs_set_material can later bind any material of up to layout_nphase phases.  Otherwise as
 * hs_create. */
hs_status hs_create_sized(hs_ctx** out, const int grid[3], const hs_material* m, const double C0[36],
                          const hs_options* opt, int layout_nphase, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Bind a context to another microstructure of the same grid, keeping its workspace, launch
 * configuration and captured iteration graphs resident (a serving slot reused for a new
 * request).  The phase ids and table are copied in (m as for hs_create; at most the phase count
 * the layout was sized for) and the reference medium is chosen again (C0, or the policy when
 * NULL).  Captured graphs stay valid when the reference medium is isotropic and the phases stay
 * isotropic (or stay anisotropic); otherwise the next solve captures them again.  Removes any
 * eigenstrain and warm-start state.
 * Errors: as hs_create.  After an error the context holds no valid material and refuses to
 * solve until a later hs_set_material succeeds. */
hs_status hs_set_material(hs_ctx* c, const hs_material* m, const double C0[36]);

/* Real-space corner displacement of the last solve's final evaluation, FP64 [3][N3][N2][N1]
 * (u_k of the corner (l+1/2, m+1/2, n+1/2) at index (l, m, n)), device pointer: the FP64
 * displacement of HS_FP32_REFINED, or the inverse transform of the state that the last
 * evaluation of HS_FP64 / HS_FP32 read (FP32 values widened). */
hs_status hs_get_displacement(hs_ctx* c, double* u);

/* Solve for one applied macroscopic strain (Algorithm 1 under strain control).
 *  E          host, 6 tensor components in Voigt order; all zero only with an eigenstrain set.
 *  tol        stop at the first evaluation with err < tol (tol = 0: run max_iter evaluations).
 *  max_iter   maximum number of residual evaluations (>= 1).  The iteration count is the
 *             number of residual evaluations: a homogeneous medium converges in 1.
 *  eps_out, sig_out  device pointers [6][N3][N2][N1] (double, or float if opt.out_f32), or NULL:
 *             eps = E + 1/2(deps^T1 + deps^T2) (tensor components), sigma = 1/2(sigma^T1+sigma^T2).
 *             The fields are written only when both pointers are given; with either NULL, neither
 *             is written (and no field pass runs).
 *  sig_eff    host, 6: <sigma> in Voigt order (the effective stress).
 *  iters      host: residual evaluations used.   final_err: host: err of the last evaluation.
 * Starts from u = 0 unless hs_set_state was called since the last solve.
 * Returns HS_OK, HS_NOT_CONVERGED (outputs written for the last iterate), HS_DIVERGED, or an
 * error. */
hs_status hs_solve(hs_ctx* c, const double E[6], double tol, int max_iter, void* eps_out,
                   void* sig_out, double sig_eff[6], int* iters, double* final_err);

/* Solve under an applied macroscopic stress (Section 2.5, Eqs. Grand_Elast_energy and
 * equi_epsilon_bar; Algorithm 1 step 6).  The macroscopic strain starts at
 * E = (lambda0)^-1 : sigma^a and, after every evaluation that does not stop, moves to
 * (lambda0)^-1 : {sigma^a + (lambda0 - <lambda>) : E - <lambda : deps> + <lambda : eps0>},
 * evaluated in the equivalent form E + (lambda0)^-1 : (sigma^a - <sigma>).
 *  S          host, 6: applied stress sigma^a in Voigt order (tensor components); all zero
 *             only with an eigenstrain set.
 *  E_out      host, 6 or NULL: the macroscopic strain of the last evaluation (tensor components).
 *  Other arguments, outputs and return values as for hs_solve.
 * Stopping: HS_FP64 and HS_FP32 stop on err < tol, as Algorithm 1 does (E is updated at
 * every evaluation).  HS_FP32_REFINED updates E after every FP64 residual sweep and stops
 * when err < tol and ||sigma^a - <sigma>||_F < tol * max(||sigma^a||_F, ||<sigma>||_F).
 * The update converges at the rate set by lambda0 against the effective stiffness, so
 * references far from it (very stiff inclusions with the Section 3.4 rule) need many
 * evaluations. */
hs_status hs_solve_stress(hs_ctx* c, const double S[6], double tol, int max_iter, void* eps_out,
                          void* sig_out, double sig_eff[6], double E_out[6], int* iters, double* final_err);

/* Per-phase eigenstrain eps0 (Eq. linear_elasticity: sigma = lambda(r) : (eps(r) - eps0(r))).
 *  eps0       host, nphase x 6 tensor components in Voigt order, copied; NULL removes it.
 * Applies to every later hs_solve / hs_solve_stress of this context.  Stress outputs and
 * <sigma> include -lambda : eps0; the strain output is the total strain E + deps.
 * Errors: HS_ERR_INVALID_ARG (non-finite values), HS_ERR_CUDA. */
hs_status hs_set_eigenstrain(hs_ctx* c, const double* eps0);

/* Error after each residual evaluation of the last hs_solve (HS_FP32_REFINED: the FP32
 * evaluations of its first, plain solve, then one value per FP64 residual sweep).
 * Writes min(n, available) values; *n_written gets the count. */
hs_status hs_err_history(const hs_ctx* c, double* out, int n, int* n_written);

/* Displacement state u(q) after the last solve, as complex128 [3][N3][N2][N1/2+1]
 * (interleaved re, im), device pointer.  Convention: the corner at (l+1/2, m+1/2, n+1/2)
 * carries index (l, m, n) and u(q) = 1/N sum_c u(c) exp(-i q.c), i.e. the paper's u(q) of
 * Eq. FT_u times exp(i q.(1/2,1/2,1/2)).  Not available in HS_FP32_REFINED mode. */
hs_status hs_get_state(hs_ctx* c, void* uhat);

/* Load a displacement state (same format, device pointer) as the starting point of the next
 * hs_solve (warm start / checkpoint resume).  Not available in HS_FP32_REFINED mode. */
hs_status hs_set_state(hs_ctx* c, const void* uhat);

/* The reference medium in use (host, 6x6 Voigt). */
hs_status hs_get_reference_medium(const hs_ctx* c, double C0[36]);

/* Kernel classes reported by hs_profile_read. */
enum {
  HS_K_XPASS = 0,     /* real-space pass: stencil, constitutive step, adjoint stencil (with the x FFTs
                         when xfuse = 1) */
  HS_K_YFWD = 1,      /* forward y FFT */
  HS_K_ZGREEN = 2,    /* forward z FFT, Green update, inverse z FFT */
  HS_K_YINV = 3,      /* inverse y FFT */
  HS_K_RESID64 = 4,   /* FP64 real-space residual sweep (HS_FP32_REFINED) */
  HS_K_FIELDS = 5,    /* output of eps and sigma */
  HS_K_OTHER = 6,     /* state transforms, correction accumulation, set-up */
  HS_K_XINV = 7,      /* inverse x FFT (half spectrum -> real rows), xfuse = 0 */
  HS_K_XFWD = 8,      /* forward x FFT (real rows -> half spectrum), xfuse = 0 */
  HS_K_XPASS_SRC = 9, /* real-space pass of a correction solve (reads the FP32 correction source;
                         HS_FP32_REFINED) */
  HS_K_COUNT = 10
};

/* Start (on >= 1) or stop (on = 0) per-launch timing.  Timed launches are bracketed by CUDA
 * events on the context's stream.  on = n times the launches of one iteration chunk in every n
 * (as plain launches; the other chunks replay their captured graph as without timing) and every
 * launch outside the chunks (FP64 sweeps, field passes, set-up); on = 1 times every launch.  The
 * events add a few microseconds of host work and a short gap on the device per timed launch.
 * Errors: HS_ERR_INVALID_ARG for on < 0. */
hs_status hs_profile_enable(hs_ctx* c, int on);

/* Device time (ms, from the events) and launch counts per kernel class since the last read;
 * resets the accumulators.  ms and launches have HS_K_COUNT entries.  Launch counts cover every
 * kernel launched or replayed, whether or not timing is enabled; when only some launches of a
 * class were timed, ms is their total scaled by (launches / timed launches), so ms / launches is
 * the mean time of the timed launches. */
hs_status hs_profile_read(hs_ctx* c, double ms[10], long long launches[10]);

/* ---- Batched solves: many RVEs and their load cases in shared launches ----------------------
 * An item is one microstructure (RVE) under one macroscopic strain; the 6 unit strains of an RVE
 * give its effective 6x6 stiffness (Eq. final_fields, <sigma> per load case).  Items whose RVEs
 * share a grid and phase isotropy form a size class.  Every item owns a full single-solve
 * workspace (hs_workspace_size of its RVE's grid, with the class's largest phase count); the items
 * of a class lie one stride apart in the batch workspace, and every kernel of a class runs as ONE
 * launch over all its items.  A chunk of check_every iterations of every class is captured as one
 * CUDA graph (the classes on streams forked from the batch stream, so they overlap) and replayed
 * until every item has stopped.  Each item has its own status and stopping test, its own reference
 * medium (the C0 policy of hs_create) and its own error history, and the same iterates as a
 * single hs_solve of that item (reductions run in the same order). */
typedef struct hs_batch hs_batch;

/* Workspace bytes of a batch.
 *  nrve       number of RVEs; grids: host nrve x 3 (N1, N2, N3, as hs_create); nphase: host nrve.
 *  nitem      number of items; item_rve: host nitem RVE indices in 0..nrve-1 (any order; an RVE
 *             may appear several times).
 *  opt        shared options (precision; xfuse must be 0).
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_UNSUPPORTED_SIZE (a grid hs_create refuses). */
hs_status hs_batch_workspace_size(int nrve, const int* grids, const int* nphase, int nitem, const int* item_rve,
                                  const hs_options* opt, size_t* bytes);

/* Create a batch.
 *  mats       host nrve materials, ids kinds only (HS_IDS_U8 / HS_IDS_U16; compress a per-voxel
 *             field with hs_compress_coefficients first); read during this call.
 *  autotune   1: each class takes its launch shapes from hs_autotune's plan cache, tuning on the
 *             class's first workspace when the cache has no plan for that grid; 0: opt as given.
 *  workspace  device memory of at least hs_batch_workspace_size bytes, 256-byte aligned, owned by
 *             the caller, in use until hs_batch_destroy.   stream: cudaStream_t (NULL = legacy
 *             default stream, which cannot be captured: plain launches then).
 * Errors: as hs_create; HS_ERR_OOM for a small workspace. */
hs_status hs_batch_create(hs_batch** out, int nrve, const int* grids, const hs_material* mats, int nitem,
                          const int* item_rve, const hs_options* opt, int autotune, void* workspace,
                          size_t workspace_bytes, void* stream);

/* Solve every item (Algorithm 1 under strain control, in the batch's precision).
 *  E          host nitem x 6: item i's macroscopic strain (tensor components, Voigt order), not 0.
 *  tol, max_iter  as hs_solve, for every item.
 *  sig_eff    host nitem x 6: <sigma> of the last evaluation of each item.
 *  iters, final_err, status  host nitem: evaluations used, err of the last evaluation, and the
 *             hs_status each item would have from hs_solve (HS_OK, HS_NOT_CONVERGED, HS_DIVERGED).
 * HS_FP32_REFINED runs every item's stages in step: its plain FP32 first solve, then FP64
 * residual sweeps (which take every stop decision) alternating with FP32 correction solves; an
 * item that stops retires and every kernel skips it.  No fields are written.
 * Returns HS_OK when every item converged, HS_NOT_CONVERGED otherwise, or an error. */
hs_status hs_batch_solve(hs_batch* b, const double* E, double tol, int max_iter, double* sig_eff, int* iters,
                         double* final_err, int* status);

/* Error history of item `item` after the last hs_batch_solve: every evaluation (HS_FP64, HS_FP32),
 * or one value per FP64 residual sweep (HS_FP32_REFINED).  Writes min(n, available) values. */
hs_status hs_batch_err_history(const hs_batch* b, int item, double* out, int n, int* n_written);

/* Kernel launches of the batch since the last call (replayed graph nodes counted per replay). */
hs_status hs_batch_launches(hs_batch* b, long long* launches);

/* Number of size classes, and (if class_of_item is not NULL) the class of every item. */
hs_status hs_batch_classes(const hs_batch* b, int* nclass, int* class_of_item);

/* Text of the last error of this batch (or of the last failed create). */
const char* hs_batch_last_error(const hs_batch* b);

/* Release the batch (the workspace stays the caller's). */
void hs_batch_destroy(hs_batch* b);

/* Limits of hs_residual_noalloc's fixed scratch array. */
#define HS_NOALLOC_SCRATCH_BYTES (512 * 1024) /* bytes held on every device that loads the library */
#define HS_NOALLOC_MAX_PHASES 1024            /* phases the array can hold */
#define HS_NOALLOC_MAX_BLOCKS 4096            /* per-block partial sums the array can hold */

/* Equilibrium residual of a displacement field, for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a library convenience.  It is for code that must not
 * allocate at the moment it runs - real-time or embedded callers with a fixed memory budget,
 * callers whose device memory belongs entirely to another allocator (a caching pool), checks run
 * where an allocation could fail or stall - and who therefore cannot supply hs_create's
 * workspace.  It computes, in FP64, the nodal force F = dE/du (the derivative of the
 * tetrahedral-stencil elastic energy with respect to each corner displacement) at the real-space
 * corner displacement u, the mean stress <sigma> and the root mean square of F, the same values
 * the FP64 residual sweep of HS_FP32_REFINED computes.
 *  grid       N1, N2, N3: the grids hs_create accepts (even, 4..512, prime factors 2, 3, 5, 7, 11).
 *  ids        device, uint16 phase ids [N3][N2][N1]; every id must be < nphase.
 *  table      host, nphase x 36 Voigt stiffness (as hs_material.table); 1 <= nphase <= HS_NOALLOC_MAX_PHASES.
 *  E          host, macroscopic strain (tensor components, Voigt order).
 *  u          device, FP64 [3][N3][N2][N1]: u_k of the corner (l+1/2, m+1/2, n+1/2) at index (l, m, n).
 *  force      device, float [3][N3][N2][N1], or NULL.
 *  sig_mean   host, 6: <sigma> = 1/2(<sigma^T1> + <sigma^T2>).      l2: host, sqrt(1/N sum |F|^2).
 *  stream     cudaStream_t (NULL = legacy default stream); the call returns after its results are on the host.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  Its scratch is one file-scope
 * device array of HS_NOALLOC_SCRATCH_BYTES, held by every device that loads the library until the process
 * exits.  The first call on a device looks up that array's device address (with the device current), so
 * make that first call before any stream capture.  All calls share the array and each call resets what
 * must start from zero; calls that overlap on the GPU (other streams, other host threads) race on it.
 * Errors: HS_ERR_INVALID_ARG (null pointer, non-finite E or stiffness, nphase out of range, an id >= nphase,
 * checked on the device before the residual runs), HS_ERR_UNSUPPORTED_SIZE (a grid hs_create refuses, more
 * blocks than HS_NOALLOC_MAX_BLOCKS, or no row tile whose shared memory fits the device), HS_ERR_CUDA. */
hs_status hs_residual_noalloc(const int grid[3], const unsigned short* ids, const double* table, int nphase,
                              const double E[6], const double* u, float* force, double sig_mean[6],
                              double* l2, void* stream);

/* Release the context (the workspace stays the caller's). */
void hs_destroy(hs_ctx* c);

/* Static description of a status code. */
const char* hs_error_string(hs_status s);

/* Text of the last error recorded on this context ("" if none). */
const char* hs_last_error(const hs_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* HS_H */
