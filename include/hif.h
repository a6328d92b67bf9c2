/*
 * hif.h -- C ABI of the GB300 hierarchical interpolative factorization (HIF).
 *
 * Method: Li & Ying, "Distributed-memory Hierarchical Interpolative
 * Factorization" (arXiv:1607.00346).  The library factors the seven-point
 * discretisation A of
 *
 *     -div(a grad u) + b u = f          (§1, eq. 1; stencil of §2.4)
 *
 * on an n x n x n interior grid of the unit cube with zero Dirichlet
 * boundary (h = 1/(n+1); half-point coefficients are harmonic means of the
 * grid values, a_j towards the boundary), or on the periodic n^3 grid of the
 * unit torus (h = 1/n; hif_grid.bc), as A ~= F with
 *
 *     F^{-1} = W^0 ... W^{L-1} W^L D^{-1} W^{L T} ... W^{0 T}     (§2.4)
 *
 * where every W^l is the product of the level's sparse eliminations S_I
 * (§2.2) and skeletonizations Q_F S_F~ of faces and edges (§2.3).
 *
 * Conventions for every entry point:
 *   - A grid function is a double array of n^3 values, point (j1,j2,j3) at
 *     index j1 + n*j2 + n*n*j3.  nrhs right-hand sides are stored one after
 *     the other (column j at offset j*n^3).
 *   - Array pointers may point to host memory or to device memory of the
 *     current CUDA device; the library detects which and copies host data
 *     in and out itself.  The caller keeps ownership of all its arrays.
 *   - Calls are ordered on the given stream.  hif_factor synchronises the
 *     stream a few times per level (the ranks found by the interpolative
 *     decompositions decide the next level's sizes); hif_apply returns
 *     without synchronising when f and u are device pointers; hif_solve
 *     synchronises once per iteration to test convergence.
 *   - Errors are returned as hif_status, never thrown.  hif_last_error()
 *     gives a message for the calling thread's last failure.  After an error
 *     in hif_factor, *out is NULL and nothing is leaked.
 *   - A handle may be used from one thread at a time.
 */
#ifndef HIF_H_
#define HIF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hif_handle_s* hif_handle;
typedef struct CUstream_st* hif_stream;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  HIF_OK = 0,
  HIF_ERR_INVALID_ARG = 1,     /* bad size, NULL pointer, a <= 0 or NaN, n not m*2^L */
  HIF_ERR_OOM = 2,             /* device allocation failed */
  HIF_ERR_NOT_SPD = 3,         /* a Cholesky pivot was not positive */
  HIF_ERR_NO_CONVERGENCE = 4,  /* hif_solve reached max_iter */
  HIF_ERR_TIMEOUT = 5,         /* a bounded device-side wait expired */
  HIF_ERR_CUDA = 6             /* any other CUDA runtime error */
} hif_status;

/* Grid (§2.1): n = m 2^L points per dimension, leaf cells of side m. */
typedef struct {
  int n;
  int m;
  int bc;        /* 0: zero Dirichlet boundary on the n^3 interior grid,
                    h = 1/(n+1).  1: periodic, the paper's own setting (§2.1,
                    §4): grid points j/n of the unit torus, h = 1/n, every
                    multiple of the cell side a separator; the operator is
                    singular for b = 0, so b must be > 0 everywhere. */
} hif_grid;

enum { HIF_PREC_FP64 = 0, HIF_PREC_FP32 = 1 };

typedef struct {
  double eps;        /* relative precision of the ID (Table 2); 0 = no
                        skeletonization: exact nested-dissection elimination */
  int precision;     /* HIF_PREC_FP64: every factor block in double.
                        HIF_PREC_FP32: factor blocks in float; the ID of a
                        front too large for one SM's shared memory keeps its
                        column norms in double and downdates them there
                        (recomputing on cancellation), the ID of a smaller
                        front recomputes every norm from the updated entries
                        at each step in float (no downdate, nothing to
                        cancel); fronts flagged by pivot growth are
                        refactored in double (retry_growth); hif_solve keeps
                        the residual r = f - A u in double. */
  int use_graphs;    /* 1: the two sweeps of an apply (hif_apply, and the
                        preconditioner inside hif_solve) are captured once
                        per nrhs as a CUDA graph on a private stream and
                        replayed on the caller's stream; 0: launched one by
                        one */
  double pcg_tol;    /* hif_solve stops when ||r||_2 <= pcg_tol ||f||_2 */
  int max_iter;      /* hif_solve iteration limit */
  int tensor_cores;  /* HIF_PREC_FP32 only.  1: the deep products of the
                        partial Cholesky (the cell products X^T = A_NI L^-T and
                        A_NN -= X^T X, the rank-256 block updates, the large
                        triangular-inverse merges) run on the tensor cores
                        (TF32 with the 3xTF32 split, FP32 accumulation); 0:
                        every product on the FP32 FMA units.  FP64 factors
                        never use them. */
  double retry_growth; /* HIF_PREC_FP32 only: a front whose Cholesky (the
                        LDL^T of §2.2 / §2.3) meets a pivot d_j with
                        A_jj / d_j > retry_growth (A_jj its original
                        diagonal entry), or a pivot that is not positive, is
                        refactored in double and stored in float
                        (hif_stats.retried_fronts counts them); 0: no retry,
                        such a pivot fails with HIF_ERR_NOT_SPD.  Must be
                        finite and >= 0. */
} hif_options;

/* Fill *opt with defaults: eps 1e-6, FP64, graphs on, pcg_tol 1e-10, 200 its,
   tensor cores on, retry_growth 1e5. */
void hif_default_options(hif_options* opt);

/*
 * hif_factor -- build F ~= A (§2.4; level loop, then the root of level L).
 *   grid:  n, m with n = m 2^L, L >= 1, n <= 1024.
 *   a:     n^3 doubles, every value finite and > 0 (host or device).
 *   b:     n^3 doubles (host or device), or NULL to use b_const everywhere;
 *          every value finite and >= 0 (> 0 on the periodic grid).
 *   opt:   options (NULL = defaults).
 *   out:   receives the handle; the handle owns every device buffer of the
 *          factor until hif_destroy.
 * Errors: INVALID_ARG, OOM, NOT_SPD, TIMEOUT, CUDA.
 */
hif_status hif_factor(const hif_grid* grid, const double* a, const double* b,
                      double b_const, const hif_options* opt, hif_stream stream,
                      hif_handle* out);

/*
 * hif_apply -- u = F^{-1} f for nrhs right-hand sides (§2.4: the forward
 * sweep W^{0T} ... W^{(L-1)T}, the root solve, then W^{L-1} ... W^0).
 * f and u hold nrhs*n^3 doubles; they may alias (in-place apply).
 */
hif_status hif_apply(hif_handle h, const double* f, double* u, int nrhs,
                     hif_stream stream);

/*
 * hif_apply_noalloc -- the same u = F^{-1} f as hif_apply, for callers that
 * must not allocate device memory: a serving process that reserves all of
 * its memory up front, or code that runs where calling the CUDA allocator is
 * not allowed.  hif_apply allocates its work vectors on the handle's first
 * apply; this entry point allocates nothing and takes its work space from
 * one fixed 32 MiB array in device memory that the library defines (every
 * GPU that loads the library holds it until the process exits).  The paper
 * has no counterpart; it is a deployment variant of the apply.
 *   f, u:  nrhs*n^3 doubles in device memory (host pointers are rejected,
 *          since staging them would need an allocation); they may alias.
 *   Limit: the factor type's size times (n^3 + the largest sweep stage's
 *          work) per right-hand side must fit in 32 MiB (a 64^3 grid fits
 *          with up to three right-hand sides in FP64, a 128^3 grid does
 *          not fit); a larger request returns
 *          HIF_ERR_INVALID_ARG with the needed size in hif_last_error().
 *   The first call on a device looks up the array's device address on that
 *   device; make that first call before any stream capture.  Every call
 *   shares the one array, so calls whose work overlaps on the GPU race with
 *   each other; order them on one stream.  The array keeps the last call's
 *   contents; no part of it needs to start at zero, because each sweep
 *   writes every work entry before reading it.  Kernel profiling
 *   (hif_profile_begin) must be off.
 */
hif_status hif_apply_noalloc(hif_handle h, const double* f, double* u, int nrhs,
                             hif_stream stream);

/*
 * hif_residual -- r = f - A u with the handle's operator, in double.
 */
hif_status hif_residual(hif_handle h, const double* f, const double* u,
                        double* r, int nrhs, hif_stream stream);

/*
 * hif_solve -- solve A u = f by conjugate gradients preconditioned with
 * F^{-1} (replaces the GMRES of Table 2; F^{-1} is SPD).  Each column is
 * iterated until ||r||_2 <= pcg_tol ||f||_2 (residual in double).  u is
 * the output only (the iteration starts from zero).  iters and relres, when
 * not NULL, receive per column the iteration count and the final relative
 * residual (nrhs entries each, host memory).
 * Errors: NO_CONVERGENCE when a column did not converge in max_iter
 * iterations (u then holds the last iterate).
 */
hif_status hif_solve(hif_handle h, const double* f, double* u, int nrhs,
                     hif_stream stream, int* iters, double* relres);

/*
 * hif_apply_batch -- u_i = F_i^{-1} f_i for nh factors at once (a serving
 * process holding factors of different grids answers their requests
 * together; the paper has no counterpart).  The sweeps of all the factors
 * run in shared launches: at each step every factor that has a stage there
 * adds its gathers, mat-vecs and scatters to one launch per kind, the
 * backward sweep aligned at each factor's last stage.  Every factor keeps
 * its own work buffers and the arithmetic of its own apply, so u_i is bit
 * for bit what hif_apply(h[i], f[i], u[i], nrhs[i]) gives.
 *   h:     nh distinct handles of one precision, on the current device.
 *   f, u:  arrays of nh pointers; f[i], u[i] hold nrhs[i] * n_i^3 doubles
 *          (host or device, as for hif_apply).
 * Errors: INVALID_ARG (nh < 1, NULL or repeated handles, mixed precision or
 * device, nrhs < 1), OOM, CUDA.
 */
hif_status hif_apply_batch(const hif_handle* h, int nh, const double* const* f,
                           double* const* u, const int* nrhs, hif_stream stream);

/*
 * hif_solve_batch -- hif_solve for nh factors at once: the conjugate
 * gradients of all the systems advance in lockstep and every
 * preconditioner application is one hif_apply_batch of the systems still
 * iterating.  Each system's iteration is the one hif_solve runs (same
 * kernels, same scalar arithmetic, its own pcg_tol and max_iter), so its
 * u, iteration counts and residuals are bitwise those of hif_solve alone.
 * iters and relres (host, optional) receive sum(nrhs) entries, the columns
 * of the systems in order.
 * Errors: as hif_apply_batch, and NO_CONVERGENCE if any column did not
 * converge.
 */
hif_status hif_solve_batch(const hif_handle* h, int nh, const double* const* f,
                           double* const* u, const int* nrhs, hif_stream stream, int* iters,
                           double* relres);

/* Per-factorization statistics, filled by hif_query_stats. */
typedef struct {
  int n, m, levels, precision;
  double eps;
  int root_size;                 /* |Sigma^L| (Table 2) */
  int64_t active_after[16];      /* |Sigma^{l+1}| after level l */
  int64_t fronts[16][3];         /* cells, skeletonized faces, edges per level */
  double factor_seconds;         /* wall time of hif_factor */
  double level_seconds[17];      /* per level, then the root */
  double flops;                  /* algorithmic flops of the factorization */
  size_t factor_bytes;           /* device bytes held by the handle */
  size_t peak_bytes;             /* peak device bytes during hif_factor */
  int64_t stored_entries;        /* factor entries read by one apply sweep */
  int kernel_launches;           /* kernels launched by hif_factor */
  int apply_launches;            /* kernels launched by one hif_apply (nrhs = 1) */
  int64_t retried_fronts;        /* FP32 fronts refactored in double (retry_growth) */
} hif_stats;

hif_status hif_query_stats(hif_handle h, hif_stats* st);

/*
 * hif_query_active -- the DOFs still active after level `level` (Sigma^{l+1}
 * of §2.4: what the level's cell eliminations and the interpolative
 * decompositions of its faces and edges kept), as sorted grid indices in
 * host memory.  level = L-1 gives the root set Sigma^L.  Call it with
 * out = NULL to get *count, then again with cap >= *count.
 * Errors: INVALID_ARG (NULL handle or count, level outside [0, L), cap too
 * small).
 */
hif_status hif_query_active(hif_handle h, int level, int32_t* out, int64_t cap,
                            int64_t* count);

/*
 * hif_predict_bytes -- device bytes hif_factor is expected to need at its
 * peak for this grid and options (used for admission control): an upper
 * estimate fitted to measured peaks (within ~25-60% above them at eps 1e-6
 * to 1e-4 for n = 64 ... 256); it depends on n, the precision and eps, not
 * on the coefficients.  0 for an invalid grid.
 */
size_t hif_predict_bytes(const hif_grid* grid, const hif_options* opt);

/*
 * Kernel profiling.  hif_profile_begin() clears the record and starts timing
 * every kernel the library launches (CUDA events on the launching stream);
 * hif_profile_end() stops, waits for the recorded events and writes up to
 * cap per-kernel aggregates (*count receives the number available).  flops
 * and bytes are the algorithmic counts of the launches (0 where not defined).
 * An apply whose sweeps replay a CUDA graph is timed as one launch named
 * "apply_sweeps_graph" (its kernels are not timed one by one).
 * Process-wide; meant for benchmarking, not for concurrent use.
 */
typedef struct {
  char name[48];
  int64_t launches;    /* timed launches (a CUDA graph replay counts as one) */
  int64_t kernels;     /* kernels those launches ran (a replay runs many) */
  double seconds;
  double flops;
  double bytes;
} hif_kernel_profile;

hif_status hif_profile_begin(void);
hif_status hif_profile_end(hif_kernel_profile* out, int cap, int* count);

/*
 * Autotuning of the launch shapes (the paper has no counterpart: its dense
 * algebra is Elemental's).  Two kernels have shapes that do not change a
 * single bit of any result but decide their speed: the cluster pivoted QR of
 * the large IDs (CTAs per front, 1-16, and how many fronts share a launch:
 * all at once, or as many as fit the L2 cache) and the tensor-core products
 * (K chunk and tile width).  Fronts and products are put into size buckets
 * (ID: front width x number of fronts; products: rows, width and depth of
 * the batch x waves of tiles).
 *
 * hif_autotune -- factor the given operator once while measuring: every
 * cluster ID without a table entry times its candidate shapes in place on
 * copies of its own matrices; the tensor-core products record their
 * shapes, which are then replayed with every tile variant.  The fastest
 * shape per bucket is kept process-wide and used by every later hif_factor
 * (the built-in rule elsewhere).  Arguments as for hif_factor; path: a
 * table file to write (NULL: none); with force = 0 and a readable table for
 * this device at path, the table is loaded instead of measured.
 * hif_autotune_load reads such a file (INVALID_ARG if it is malformed or
 * was written for another device), hif_autotune_clear returns to the
 * built-in rules, hif_autotune_table copies the current table as text
 * (*len = its length; buf may be NULL).
 */
hif_status hif_autotune(const hif_grid* grid, const double* a, const double* b, double b_const,
                        const hif_options* opt, const char* path, int force, hif_stream stream);
hif_status hif_autotune_load(const char* path);
void hif_autotune_clear(void);
hif_status hif_autotune_table(char* buf, size_t cap, size_t* len);

/* Release every resource of the handle (NULL is ignored). */
void hif_destroy(hif_handle h);

/*
 * hif_save / hif_load -- factor persistence (no counterpart in the paper: a
 * serving process keeps factored operators across restarts).
 *   hif_save writes the handle's factor (every stage's device arrays and
 *   mat-vec lists, the operator, options and statistics) to `path`, a
 *   versioned binary file; it synchronises the device first.
 *   hif_load reads such a file into a new handle (*out; NULL on error); the
 *   handle applies and solves exactly as the saved one (bitwise the same
 *   results).  Files are read only by the build that wrote them (the
 *   option and statistics layouts are checked).
 *   hif_load checks every count, index and mat-vec extent of the file
 *   against the sizes of the arrays it read (and the apply work stride
 *   against the stage lists) before any kernel can use them.
 * Errors: INVALID_ARG (NULL arguments, unreadable or unwritable path, not a
 * factor file, another version, truncated or corrupt file, inconsistent
 * contents), OOM, CUDA.
 */
hif_status hif_save(hif_handle h, const char* path);
hif_status hif_load(const char* path, hif_handle* out);

/* Message for the calling thread's last failed call ("" if none). */
const char* hif_last_error(void);

/* Library version string. */
const char* hif_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HIF_H_ */
