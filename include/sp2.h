/*
 * sp2.h -- C ABI of a GB300 (sm_103a) library that computes the zero-temperature
 * density matrix D of a symmetric block-sparse Fock/Kohn-Sham matrix F with the
 * SP2ACC recursive expansion and error-controlled truncation.
 *
 * Paper: A. Kruchinina, E. Rudberg, E. H. Rubensson, "Efficient computation of the
 * density matrix with error control on distributed computer systems",
 * arXiv:1909.12533.  Section 1 defines D (Eq. (3): projector onto the nocc lowest
 * eigenvectors of F); Section 4 gives the method: Step 1 (schedule, Gershgorin
 * bounds, Algorithm 1), Step 2 (Algorithm 2: X_i = ((1-a)I + a X~)^2 or
 * 2aX~ - (aX~)^2, truncation X~_i = X_i + E_i, e_i = ||X~_i - X~_i^2||_F,
 * t_i = trace(X~_i - X~_i^2), parameterless stop with C = 6.8872), Step 3
 * (homo/lumo estimates from e_i and t_i).  Section 2 gives the truncation error
 * control (Eqs. (6)-(8)), Section 3 the Frob-Inf norm (Eq. (13)).
 *
 * Conventions (all entry points):
 *  - Every function returns SP2_OK (0) or a negative SP2_ERR_* code; no C++
 *    exception crosses this boundary.  sp2_strerror() names a code.
 *  - Matrices are exchanged as sp2_bsr: tiles of b x b with b = 32, only tiles
 *    with block row <= block column stored, sorted by (row, col), values
 *    row-major inside each tile, diagonal tiles stored in full (both triangles),
 *    every diagonal tile present.  When N is not a multiple of 32 the last tile
 *    row/column is zero padding and stays zero.
 *  - All GPU work is issued on the caller's CUDA stream (cudaStream_t passed as
 *    void*; NULL = legacy default stream).  Calls synchronise that stream only
 *    where they need a scalar on the host (counts, e_i / t_i for the stop test).
 *  - The context owns all device memory it allocates.  Inputs are copied;
 *    the caller keeps ownership of its buffers.
 *  - Not thread-safe per context; different contexts are independent.
 */
#ifndef SP2_H
#define SP2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define SP2_OK                 0
#define SP2_ERR_INVALID_ARG   -1  /* NULL pointer, bad size, b != 32, bad enum     */
#define SP2_ERR_BOUNDS        -2  /* homo_ub >= lumo_lb, or bounds outside [lmin, lmax] */
#define SP2_ERR_PATTERN       -3  /* tiles unsorted, lower-triangle, out of range, missing diagonal tile */
#define SP2_ERR_NONFINITE     -4  /* NaN or Inf in F (or W)                        */
#define SP2_ERR_OOM           -5  /* device allocation failed                      */
#define SP2_ERR_CUDA          -6  /* a CUDA runtime call failed                    */
#define SP2_ERR_NOT_CONVERGED -7  /* n_max reached without the stop test firing; D is still readable */
#define SP2_ERR_TIMEOUT       -8  /* a bounded device wait gave up                 */
#define SP2_ERR_STATE         -9  /* call out of order (e.g. get_D before run)     */
#define SP2_ERR_CAPACITY     -10  /* caller buffer too small (size returned)       */
#define SP2_ERR_TOO_LARGE    -11  /* input exceeds the fixed scratch of sp2_truncate_noalloc */
#define SP2_ERR_RANGE        -12  /* an iterate left the range of the method: an element with |x| >= 2
                                     met the tensor-core slicing, or e_i / t_i is not finite
                                     (homo/lumo bounds that do not bracket the gap, or divergence) */

#define SP2_TILE 32
#define SP2_MAX_ITER 128

/* ---------------------------------------------------------------- enums */
/* Polynomial choice: SP2 and SP2ACC follow the schedule of Section 4 Step 1
 * (homo/lumo bounds required); TRACE is the trace-correcting expansion of
 * Section 1 (p_i = 1 iff trace(X~_{i-1}) > nocc, alpha_i = 1, no bounds needed:
 * the first run of Section 6). */
enum sp2_mode      { SP2_MODE_SP2 = 0, SP2_MODE_SP2ACC = 1, SP2_MODE_TRACE = 2 };
/* Stop tests: Algorithm 2's parameterless criterion, or e_j < idem_tol. */
enum sp2_stop      { SP2_STOP_PARAMETERLESS = 0, SP2_STOP_IDEMPOTENCY = 1 };
/* Truncation norm: Frobenius (Section 2), Frob-Inf (Section 3, Eq. (13)) or the
 * Frobenius-spectral mixed norm ||.||_m of Section 3 (the spectral norm of the
 * matrix of block Frobenius norms; blocks of frobinf_part rows, at most 512
 * block rows).  MIXED: every tile whose squared norm is at most a threshold is
 * dropped, for the largest threshold whose error has a mixed-norm bound (a
 * Collatz-Wielandt bound from 100 power steps) of at most tau; found by
 * bisection with one host round trip per step. */
enum sp2_trunc     { SP2_TRUNC_FROBENIUS = 0, SP2_TRUNC_FROBINF = 1, SP2_TRUNC_MIXED = 2 };
/* Arithmetic of the tile products X~ X~:
 *   FP64   : FP64 fused multiply-adds on the CUDA cores.
 *   SPLIT16: tcgen05 tensor-core MMAs on FP16 slices of X~ on fixed absolute
 *            grids (slice s on the grid 2^-(11 s - 1)); products of slice pairs
 *            (s, t) with s + t <= slices + 1 accumulate exactly-grouped in FP32
 *            tensor memory and are combined in FP64.  slices = 2 is the
 *            hi+lo three-product form.  slices = 5 uses 10-bit slices
 *            (finest grid 2^-49, FP64 grade for |x| <= 1) and runs each square
 *            as two launches: the finest group (s + t = 6) first, its exact
 *            sum left in the output tiles, then the other four groups added
 *            to it in the full epilogue (tensor memory holds four group
 *            accumulators), every K loop in segments of 8 K tiles; it does
 *            not record masks for sp2_backward.  In every slice count the
 *            diagonal of S (the squared row norms of X~) is taken in FP64.
 * Everything else (traces, norms, polynomial choice, stop test, truncation)
 * is FP64 in every precision. */
enum sp2_precision { SP2_PREC_FP64 = 0, SP2_PREC_SPLIT16 = 1 };
/* Storage of the iterates (Section 5): SYMMETRIC keeps the upper tiles only and
 * computes only the upper output tiles of each square; GENERAL keeps and
 * computes both triangles, like the paper's general-matrix implementation (the
 * comparison of Section 6).  The truncation selection is the same in both, so
 * D is the same; D is returned as upper tiles in both. */
enum sp2_storage   { SP2_STORAGE_SYMMETRIC = 0, SP2_STORAGE_GENERAL = 1 };

typedef struct {
  int64_t n;              /* matrix dimension N                                  */
  int32_t b;              /* tile size; must be 32                               */
  int64_t nnzb;           /* number of stored tiles                              */
  const int32_t* brow;    /* [nnzb] tile row I                                   */
  const int32_t* bcol;    /* [nnzb] tile column J >= I                           */
  const double* val;      /* [nnzb * b * b] tile values, row-major per tile      */
  int32_t on_device;      /* 1: the three pointers are device pointers; 0: host  */
} sp2_bsr;

/* Optional device allocator.  alloc returns NULL on failure (-> SP2_ERR_OOM).
 * NULL allocator = stream-ordered allocation (cudaMallocFromPoolAsync /
 * cudaFreeAsync on the context's stream) from a memory pool the library keeps
 * per device: memory a destroyed context freed is reused by the next context
 * without going back to the driver; sp2_release_memory() returns it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} sp2_allocator;

typedef struct {
  int32_t mode;            /* sp2_mode, default SP2ACC                                  */
  int32_t stop;            /* sp2_stop, default PARAMETERLESS                           */
  double idem_tol;         /* threshold of the idempotency stop, default 1e-12          */
  int32_t trunc;           /* sp2_trunc, default FROBENIUS                              */
  int64_t frobinf_part;    /* Frob-Inf and mixed-norm partition size in rows, multiple of 32;
                              default 4096 (Section 6)                                  */
  double gamma;            /* > 0: tau_i from Eq. (7) with this gamma; tau argument ignored */
  double delta_acc;        /* acceleration switches off once max distance <= delta_acc; default 0.1 */
  int32_t n_max_cap;       /* cap on n_max, <= SP2_MAX_ITER - 2; default 100             */
  int32_t precision;       /* sp2_precision, default FP64                               */
  int32_t slices;          /* SPLIT16 slices, 2..5, default 4                            */
  int32_t mixed_from;      /* first iteration i whose square uses `precision` (earlier ones FP64); default 1 */
  int32_t mixed_until;     /* last iteration using `precision` (later ones FP64); 0 = no limit */
  int32_t ckpt_every;      /* adjoint checkpoint interval k (X~_i kept for i % k == 0); default 8 */
  int32_t record_masks;    /* 1: keep per-iteration tile masks and FP64 checkpoints (needed by
                              sp2_backward; memory grows by one X~ per ckpt_every steps); default 0 */
  double fp64_tail;        /* SPLIT16 with the idempotency stop: once e_j < fp64_tail, and in any case
                              for the last four squares up to n_max + 1, the squares run in
                              FP64, so the final idempotency steps reach FP64 accuracy;
                              0 = never; default 1e-4                                   */
  int32_t acc_flush_min;   /* SPLIT16: a 128 x 128 output block whose product has at least this many
                              K tiles adds its FP32 tensor-memory sums into the exact fixed-point
                              total every 16 K tiles (keeps the sums exact for dense operands);
                              0 = never; default 512                                    */
  int32_t wait_limit_ms;   /* every bounded wait inside a tensor-core kernel gives up after this
                              many milliseconds with SP2_ERR_TIMEOUT; default 2000      */
  int32_t selftest;        /* tests of the error paths (no fault, no data touched); default 0.
                              1: in the first sp2_run of the context the first tensor-core square
                              waits, before it moves any data, on a barrier that nothing arrives
                              at; the wait gives up after wait_limit_ms and sp2_run returns
                              SP2_ERR_TIMEOUT.  2: in the first sp2_run the first slicing of a
                              tensor-core operand reports an out-of-range element (its data are
                              unchanged) and sp2_run returns SP2_ERR_RANGE.  Later runs of the
                              context are unaffected.                                   */
  int32_t storage;         /* sp2_storage, default SYMMETRIC; GENERAL does not record masks for
                              sp2_backward (record_masks must be 0)                    */
  int32_t split_supply;    /* SPLIT16: 1 = the B operand slices of the tensor-core square reach
                              shared memory through two copy warps (16-byte cp.async) while
                              the A slices come by bulk copy; 0 = bulk copies only.  Same
                              results either way; default 0                            */
} sp2_params;

typedef struct {
  int32_t status;          /* return code of the last sp2_run                          */
  int32_t converged;       /* 1 when the stop test fired                               */
  int32_t n;               /* index n of the returned iterate X~_n                     */
  int32_t n_min, n_max;    /* schedule (Section 4, Step 1)                             */
  int32_t squares;         /* matrix squares computed (n + 1)                          */
  double lmin, lmax;       /* Gershgorin bounds (Algorithm 1)                          */
  double homo_est, lumo_est; /* Step 3 estimates (NaN when unavailable)                 */
  int32_t have_estimates;  /* bit 0: homo_est valid, bit 1: lumo_est valid */
  int64_t nnzb_final;      /* stored tiles of D                                        */
  int64_t tile_triplets;   /* sum over squares of the (I <= J, K) tile triplets computed
                              (GENERAL storage: all (I, J, K) of both triangles)        */
  double alg_flops;        /* 2 * 32^3 * tile_triplets                                 */
  double run_ms;           /* device time of sp2_run (cudaEvents)                      */
  double square_ms;        /* device time spent in the tile-product kernels            */
  int32_t p[SP2_MAX_ITER];        /* p_i, i = 1..n_max (p[0] unused = -1)              */
  double alpha[SP2_MAX_ITER];     /* alpha_i                                           */
  double tau[SP2_MAX_ITER];       /* tau_i, i = 0..n_max                               */
  double e[SP2_MAX_ITER];         /* e_j, j = 0..n                                     */
  double t[SP2_MAX_ITER];         /* t_j                                               */
  int64_t nnzb_hist[SP2_MAX_ITER]; /* stored tiles of X~_j                             */
  int32_t prec_hist[SP2_MAX_ITER]; /* precision of the square that produced e_j         */
  int64_t kernel_launches;        /* kernels this library launched during sp2_run      */
  double backward_ms;             /* device time of the last sp2_backward              */
  double tc_hw_flops;             /* tensor-core MMA flops issued in sp2_run (slice pairs,
                                     zero padding of 128 x 128 super-tiles included)    */
} sp2_stats;

typedef struct sp2_ctx sp2_ctx;

/* Fill *p with the defaults listed above. */
int sp2_default_params(sp2_params* p);

/* Step 1 of Section 4 (and Algorithm 1): copy F to the device, compute the
 * Gershgorin bounds lmin <= lambda_1, lmax >= lambda_N, build the schedule
 * (p_i, alpha_i, n_min, n_max, tau_i) from homo_ub >= lambda_homo and
 * lumo_lb <= lambda_lumo, form X_0 = (lmax I - F)/(lmax - lmin) and its
 * truncation X~_0.  tau is the truncation threshold of every iteration
 * (ignored when params->gamma > 0).  nocc is used for reporting only, except
 * in SP2_MODE_TRACE, where it steers the polynomial choice; that mode takes no
 * bounds (homo_ub and lumo_lb are ignored and may be NaN), n_max is n_max_cap,
 * and gamma must be 0 (Eq. (7) needs a gap bound).
 * Errors: INVALID_ARG, PATTERN, NONFINITE, BOUNDS, OOM, CUDA.  On error *out is NULL. */
int sp2_create(const sp2_bsr* F, int64_t nocc, double homo_ub, double lumo_lb, double tau,
               const sp2_params* params, const sp2_allocator* alloc, void* cuda_stream,
               sp2_ctx** out);

/* sp2_create for a dense F (Section 1: F is the N x N Fock/Kohn-Sham matrix;
 * Algorithm 1 takes it as it is).  F: n x n, row-major with leading dimension
 * ld >= n (in doubles), host or device memory per on_device; it must be
 * symmetric.  Only the tiles on and above the block diagonal are read (the
 * 32 x 32 tiles (I, J), I <= J; the diagonal tiles in full); the tiles that
 * are exactly zero are left out of the stored pattern, the diagonal tiles are
 * always kept.  The dense matrix is tiled on the device (a temporary copy of F
 * is made with the context's allocator when F is on the host); the caller
 * keeps ownership of F.  Other arguments and errors as sp2_create. */
int sp2_create_dense(const double* F, int64_t n, int64_t ld, int32_t on_device, int64_t nocc, double homo_ub,
                     double lumo_lb, double tau, const sp2_params* params, const sp2_allocator* alloc,
                     void* cuda_stream, sp2_ctx** out);

/* Step 2 of Section 4 (Algorithm 2) and Step 3: iterate until the stop test
 * fires, then estimate homo/lumo.  Returns SP2_OK, SP2_ERR_NOT_CONVERGED (D is
 * the last iterate and readable), or an error.  stats may be NULL. */
int sp2_run(sp2_ctx* ctx, sp2_stats* stats);

/* Section 6's second run: homo/lumo bounds from the Step 3 estimates of the
 * last sp2_run of ctx (typically a SP2_MODE_TRACE run).  The estimates are not
 * bounds, so each moves away from the gap by margin * (lumo_est - homo_est)
 * (the paper gives no margin; 0 <= margin < 0.5) and stays inside the
 * Gershgorin interval [lmin, lmax]:
 *   *homo_ub = max(homo_est + d, lmin),  *lumo_lb = min(lumo_est - d, lmax).
 * Errors: INVALID_ARG, STATE (no run, or the run gave no estimate of one side,
 * or lumo_est <= homo_est). */
int sp2_estimate_bounds(const sp2_ctx* ctx, double margin, double* homo_ub, double* lumo_lb);

/* Borrowed device view of D (tile arrays owned by ctx, valid until the next
 * sp2_run, sp2_backward or sp2_destroy).  view->on_device = 1. */
int sp2_get_D(sp2_ctx* ctx, sp2_bsr* view);

/* Copy D's tiles to caller buffers (host or device per `on_device`).  If
 * cap_nnzb is smaller than D's tile count, nothing is copied, *nnzb_out is set
 * and SP2_ERR_CAPACITY returned. */
int sp2_copy_D(sp2_ctx* ctx, int32_t* brow, int32_t* bcol, double* val, int64_t cap_nnzb,
               int32_t on_device, int64_t* nnzb_out);

/* D as a dense n x n matrix (both triangles; Section 1, Eq. (3): D is the
 * projector onto the occupied subspace) written to out, row-major with leading
 * dimension ld >= n (in doubles), host or device memory per on_device; the
 * caller owns out.  The entries outside D's stored tiles are written as zero.
 * The dense matrix is assembled on the device (a temporary n x n buffer from
 * the context's allocator when out is on the host).  Synchronises the stream.
 * Errors: INVALID_ARG, STATE (no D yet), OOM, CUDA. */
int sp2_copy_D_dense(sp2_ctx* ctx, double* out, int64_t ld, int32_t on_device);

/* Reverse-mode derivative of L = trace(D W) (not in the paper): W symmetric,
 * given on any tile pattern (only tiles of D's pattern matter).  Writes
 * dF = dL/dF on F's tile pattern (F's brow/bcol order; entries F_ij and F_ji
 * treated as independent, so a symmetric perturbation of an off-diagonal pair
 * changes L by 2 h dF_ij) into a borrowed device view (same lifetime rules as
 * sp2_get_D).  The iterates are recomputed from checkpoints every ckpt_every
 * steps with the recorded truncation masks.  Requires record_masks = 1. */
int sp2_backward(sp2_ctx* ctx, const sp2_bsr* W, sp2_bsr* dF_view);

/* Truncation step of Algorithm 2 as a standalone call (Section 2, Eq. (8):
 * X~ = X + E with ||E|| <= tau; Frob-Inf norm of Section 3, Eq. (13)).  X: the
 * stored upper tiles of a symmetric matrix (host or device per X->on_device;
 * X is not modified).  Tiles are ranked by (||X_IJ||_F^2, I * nb + J) and the
 * longest ascending prefix whose squared norms (weight 2 for mirrored tiles)
 * fit into tau^2 is dropped -- per Frob-Inf super-block with the budget
 * tau / max(m_R, m_C) in FROBINF mode (frobinf_part rows, multiple of 32).
 * Budget sums are exact integers in units of budget * 2^-36 (shares rounded
 * up).  keep[nnzb] (same residency as X) receives 1 = kept, 0 = dropped.
 * MIXED mode (the mixed norm of Section 3) uses the threshold rule described
 * at sp2_trunc.  Allocates its scratch with cudaMallocAsync on cuda_stream and
 * synchronises that stream before returning.  Errors: INVALID_ARG, OOM, CUDA. */
int sp2_truncate(const sp2_bsr* X, double tau, int32_t mode, int64_t frobinf_part, int32_t* keep,
                 void* cuda_stream);

/* Allocation-free variant of sp2_truncate, for callers that may not allocate
 * device memory: code that issues work while a CUDA graph is being captured,
 * callbacks of frameworks that own all device memory, or processes whose
 * allocator is locked after start-up.  (The paper has no counterpart; the
 * selection rule is that of sp2_truncate.)  All pointers are device pointers
 * that the caller owns: brow, bcol, val as in sp2_bsr (n is the matrix
 * dimension, nnzb the tile count, tiles sorted upper-triangle) and keep[nnzb]
 * for the result (1 = kept).  Work is queued on cuda_stream and not
 * synchronised.
 * Scratch: one file-scope device array of 8 MiB in this library.  Every GPU
 * that loads the library holds its own copy until the process exits, and all
 * calls on that GPU share it.  Limits: nnzb <= 262144 tiles and, in Frob-Inf
 * mode, at most 32 x 32 super-blocks (and the selection's work area must fit
 * into the array); larger inputs return SP2_ERR_TOO_LARGE.  The first call on a
 * device looks the array's device address up (cudaGetSymbolAddress) with that
 * device current and keeps it; make that first call before any stream capture.
 * A cudaDeviceReset of the device invalidates the kept address: do not call
 * this entry point on a device after resetting it.  The array keeps the
 * previous call's contents; everything that must start at zero is cleared
 * inside the call.  Calls on the same device that overlap on the GPU (for
 * example queued on two streams) race on that device's array: serialise them.
 * No cudaMalloc, cudaFree or other allocating routine is called.  Modes
 * FROBENIUS and FROBINF only (MIXED returns SP2_ERR_INVALID_ARG).
 * Errors: INVALID_ARG, TOO_LARGE, CUDA. */
int sp2_truncate_noalloc(const int32_t* brow, const int32_t* bcol, const double* val, int64_t n, int64_t nnzb,
                         double tau, int32_t mode, int64_t frobinf_part, int32_t* keep, void* cuda_stream);

int sp2_get_stats(const sp2_ctx* ctx, sp2_stats* stats);
void sp2_destroy(sp2_ctx* ctx);
const char* sp2_strerror(int code);

/* Not in the paper: hand the device memory cached by the library's memory
 * pools (memory of destroyed contexts, kept for reuse) and its cached
 * page-locked host blocks back to the driver, after the work queued on every
 * device has finished.  Contexts alive keep their memory.  Errors: CUDA. */
int sp2_release_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* SP2_H */
