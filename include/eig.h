/*
 * eig.h -- C ABI of the GB300 (sm_103a) hybrid sparse eigensolver library (libeig.so).
 *
 * Computes the n_ev algebraically smallest eigenpairs of a large sparse symmetric H
 * stored as its upper triangle (Alperen, Aktulga, Maris, Yang, "Hybrid Eigensolvers for
 * Nuclear Configuration Interaction Calculations", arXiv 2305.15552; Sec. 2 defines the
 * problem, Sec. 3.1 the half-stored matrices).
 *
 * Conventions shared by every entry point
 *   - All sizes are in elements.  Blocks of vectors are row-major n x k arrays (row i holds
 *     the k entries x_i1..x_ik contiguously); leading dimension = k unless stated.
 *   - "device" pointers are CUDA global-memory pointers of the current device; "host"
 *     pointers are ordinary CPU memory.  The library never frees caller memory and never
 *     keeps a caller pointer after a call returns, except where a handle documents it.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *     enqueued on it; calls that must read results back synchronise that stream only.
 *   - Errors: every call returns eig_status.  EIG_EINVAL for bad arguments (nothing is
 *     launched), EIG_ECUDA when a CUDA call failed (eig_last_cuda_error() gives the CUDA
 *     message), EIG_ENOMEM when device allocation failed.  A failed call leaves caller
 *     buffers in an unspecified state but never corrupts a handle.
 *   - No CPU fallback: every arithmetic step runs in this library's CUDA kernels.
 */
#ifndef EIG_H_
#define EIG_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define EIG_API __attribute__((visibility("default")))
#else
#define EIG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EIG_OK = 0,
  EIG_EINVAL = 1,          /* invalid argument (sizes, pointers, CSR structure)            */
  EIG_ENOMEM = 2,          /* device allocation failed                                     */
  EIG_ECUDA = 3,           /* a CUDA runtime call or kernel launch failed                  */
  EIG_ENOT_CONVERGED = 4,  /* maxiter reached; eig_ritz still returns the best pairs       */
  EIG_EBREAKDOWN = 5,      /* CholeskyQR / Rayleigh-Ritz basis numerically rank deficient  */
  EIG_ETIMEOUT = 6,        /* a bounded device-side wait gave up                           */
  EIG_EDUPLICATE = 7,      /* two returned eigenpairs collapsed onto the same eigenvector  */
  EIG_EUNSUPPORTED = 8     /* valid request this build does not implement (e.g. a k > max) */
} eig_status;

typedef enum { EIG_F64 = 0, EIG_F32 = 1, EIG_BF16 = 2 } eig_dtype;

typedef enum {
  EIG_LANCZOS = 0,         /* Sec. 2.1, Eqs. (krylov)-(ritzest1)                          */
  EIG_BLOCK_LANCZOS = 1,   /* Alg. 1                                                      */
  EIG_LOBPCG = 2,          /* Alg. 2                                                      */
  EIG_CHEBFILTER = 3,      /* Alg. 3 (ChebFSI)                                            */
  EIG_RMMDIIS = 4,         /* Alg. 4, batched over eigenvectors (Sec. 4.3)                */
  EIG_HYBRID = 5           /* Sec. 2.8 / Sec. 4: front method, then batched RMM-DIIS      */
} eig_method;

/* Device layout of an SpMM plan's copy of H (all compute the same Y = H X).
 * MIRRORED: the plan expands the stored triangle into both triangles on the device (8-row
 *   groups of 64-column tiles, 1-byte column indices); the kernel only gathers.  About twice
 *   the matrix bytes of HALF, and the fastest on sm_103a.
 * HALF: the stored triangle only (tile chunks); each stored entry is applied as both H_ij and
 *   H_ji, the transposed half through per-tile scratch and a fixed-order reduction.
 * CSR: the CSR copy itself, read by a reference kernel (no tiled copy is built).
 * AUTO: MIRRORED when the device has room for it while it is built, else HALF. */
typedef enum {
  EIG_LAYOUT_AUTO = 0,
  EIG_LAYOUT_MIRRORED = 1,
  EIG_LAYOUT_HALF = 2,
  EIG_LAYOUT_CSR = 3
} eig_layout;

/* Upper triangle (incl. diagonal) of a symmetric n x n matrix, CSR.
 * rowptr: int64[n+1], rowptr[0] = 0, non-decreasing; col: int32[nnz], within a row strictly
 * increasing and >= the row index (upper triangle); val: nnz values of val_type
 * (EIG_BF16 = uint16 bfloat16 bit patterns).  on_device selects host or device pointers. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t* rowptr;
  const int32_t* col;
  const void* val;
  eig_dtype val_type;
  int on_device;
} eig_csr_upper;

/* ------------------------------------------------------------------------------------ *
 * Library                                                                              *
 * ------------------------------------------------------------------------------------ */

/* Human-readable name of a status code (static string). */
EIG_API const char* eig_strerror(eig_status s);
/* Message of the last CUDA error seen by this library on the calling thread ("" if none). */
EIG_API const char* eig_last_cuda_error(void);
/* Version string of the build, e.g. "0.1.0 sm_103a". */
EIG_API const char* eig_version(void);
/* Number of CUDA kernel launches this library has made in this process (all threads). */
EIG_API int64_t eig_launch_count(void);

/* ------------------------------------------------------------------------------------ *
 * Step-level entry points (device pointers) -- one per hot-path step                    *
 * ------------------------------------------------------------------------------------ */

/* Symmetric half-stored SpMM plan.
 * The product Y = H X of Sec. 1 / Eqs. (upd1)-(upd2) with H given by its upper triangle U:
 * Y = U X + U_strict^T X, each stored off-diagonal h_ij applied as both H_ij and H_ji.
 * The plan copies H to device memory it owns (when H->on_device = 0, or always when
 * copy = 1) and builds the tile lists and the transpose schedule of the atomic-free
 * scatter: rows are grouped in row blocks of `row_block` rows (multiple of 32, <= 512),
 * columns in column blocks of `col_block` columns (multiple of 32, <= row_block, dividing
 * row_block).  0 selects defaults (256, 64); the mirrored layout needs exactly (256, 64).
 * `layout` is an eig_layout; the layout actually built is reported by eig_spmm_plan_info
 * (AUTO, or MIRRORED with other block sizes, falls back to HALF).  When copy = 0 and H is on
 * the device the plan keeps H's pointers, which must then outlive the plan.
 * Errors: EIG_EINVAL if the CSR is malformed (checked on device: sortedness, col >= row,
 * col < n) or layout is unknown, EIG_ENOMEM, EIG_ECUDA. */
EIG_API eig_status eig_spmm_plan_create_ex(const eig_csr_upper* H, int row_block, int col_block, int layout,
                                           int copy, void* stream, void** plan);
/* eig_spmm_plan_create_ex with layout = EIG_LAYOUT_AUTO. */
EIG_API eig_status eig_spmm_plan_create(const eig_csr_upper* H, int row_block, int col_block, int copy,
                                void* stream, void** plan);
EIG_API void eig_spmm_plan_destroy(void* plan);

typedef struct {
  int64_t n, nnz;
  int row_block, col_block;
  int64_t n_row_blocks, n_col_blocks;
  int64_t n_tiles;          /* nonempty (row block, column block) pairs                   */
  int64_t n_slots;          /* tiles whose transposed part goes through scratch            */
  int64_t scratch_bytes_per_col;  /* scratch bytes per vector column per byte of element    */
  eig_dtype val_type;
  int layout;               /* eig_layout the kernels run on                               */
  int64_t layout_entries;   /* entries the layout's kernel streams per product (with padding) */
  int64_t device_bytes;     /* device bytes of the plan's copies of H                      */
} eig_spmm_info;
EIG_API eig_status eig_spmm_plan_info(const void* plan, eig_spmm_info* info);

/* Y = H X.  X, Y: device, row-major n x nb, element type vec_type (EIG_F32 or EIG_F64),
 * nb in {1, 2, 4, 8, 16, 32}, both aligned to min(16, nb * element size) bytes (EIG_EINVAL
 * otherwise).  X and Y must not overlap.  Scratch for the transposed
 * partial products is owned by the plan (grown on demand; the first call for a given
 * (nb, vec_type) may allocate).  Deterministic: results are bitwise reproducible.
 * Arithmetic: FP32 vectors in FP32; FP64 vectors with FP64 values in FP64; FP64 vectors with
 * FP32 or BF16 values in the mirrored layout in double-float (exact FP32 products summed as two FP32
 * words, ~2^-44 relative per step), which sm_103a runs at FP32 rate.
 * Supported (matrix, vector) types: (F32,F32), (F64,F64), (BF16,F32), (F32,F64), (BF16,F64). */
EIG_API eig_status eig_spmm(void* plan, const void* X, void* Y, int nb, eig_dtype vec_type, void* stream);

/* One step of the Chebyshev recurrence (Alg. 3, Eq. chebypoly) fused into the product's epilogue:
 * Y = alpha (H X - c X) - Qp, or Y = alpha (H X - c X) when first != 0 (Qp unused), and Y = X on
 * columns with active[j] == 0 (device int[nb]; locked columns).  The same double arithmetic on
 * the same rounded H X as the product followed by a separate elementwise pass, with one read of X,
 * Qp and one write of Y.  Mirrored layout, nb = 8, 16 or 32, FP32 vectors with FP32 values or
 * FP64 vectors with FP64 / FP32 values; other cases return EIG_EUNSUPPORTED (compute H X with
 * eig_spmm and the step separately).  Alignment rule of eig_spmm. */
EIG_API eig_status eig_spmm_cheb(void* plan, const void* X, void* Y, int nb, eig_dtype vec_type, const void* Qp,
                                 const int* active, double alpha, double c, int first, void* stream);

/* Gram product G = A^T B (Eq. rreig's S^T S / S^T H S; Eq. bgs's V^T W).  A, B: device, row-major
 * n x nb of vec_type (F32 or F64), nb <= 64; G: device FP64 nb x nb (row-major).  FP32 inputs:
 * products in FP32, 32-row partial sums accumulated in double-float (two FP32 words), CTA
 * partials in FP64, fixed-order reduction (bitwise reproducible).  Per-call scratch is taken
 * stream-ordered (cudaMallocAsync) and released on the same stream. */
EIG_API eig_status eig_gram(const void* A, const void* B, int64_t n, int nb, eig_dtype vec_type, double* G,
                            void* stream);

/* G = A^T B as eig_gram, but without allocating device memory.  For callers that cannot
 * allocate while they run -- a framework that has reserved the whole device memory for its own
 * pool, or a latency-critical path that must not enter the driver's allocator.  The per-CTA
 * partial sums live in a file-scope __device__ array of 4 MiB (512 partials of a 32 x 32 Gram)
 * that every device loading this library holds until the process exits.  The result is
 * bitwise equal to eig_gram's while eig_gram's grid (2 CTAs per SM) fits the 512 partials --
 * always on GB300 (304); on a larger GPU the rows are grouped into 512 partials and the sums
 * round in another order.  nb <= 32, else EIG_EINVAL.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be serialised by the
 * caller.  The array is overwritten completely by each call, so nothing needs clearing.
 * The paper has no counterpart to this entry point. */
EIG_API eig_status eig_gram_noalloc(const void* A, const void* B, int64_t n, int nb, eig_dtype vec_type,
                                    double* G, void* stream);

/* eig_gram_noalloc with the CTA partials capped at max_parts (1..512, else EIG_EINVAL): the
 * grouping a GPU with more than 256 SMs would get, for checking that path on this one. */
EIG_API eig_status eig_gram_noalloc_parts(const void* A, const void* B, int64_t n, int nb, eig_dtype vec_type,
                                          double* G, int max_parts, void* stream);

/* CholeskyQR2 (Alg. 3 "CholeskyQR"; applied twice): X (device, n x k, vec_type, in place) becomes
 * Q with X_in = Q R, R (device FP64 k x k, upper triangular) = R2 R1.  k <= 64.  Returns
 * EIG_EBREAKDOWN when a squared Cholesky pivot falls below 1e-14 * max diag of the Gram
 * (X numerically rank deficient); X is then left partially updated. */
EIG_API eig_status eig_cholqr2(void* X, int64_t n, int k, eig_dtype vec_type, double* R, void* stream);

/* Lowest m eigenpairs of the symmetric k x k matrix A (device FP64, row-major; only its
 * symmetric part is used): w[m] ascending, Z (k x m row-major, orthonormal columns).  The
 * projected problems of Alg. 1 ("T U = U Theta"), Alg. 3 ("T S = S Theta").  k <= 1024,
 * m <= min(k, 256).  Householder tridiagonalisation, bisection, inverse iteration (FP64). */
EIG_API eig_status eig_small_syev(const double* A, int k, int m, double* w, double* Z, void* stream);

/* Rayleigh-Ritz on the pencil (A, G) = (S^T H S, S^T S) of Eq. (rreig): the nb leftmost
 * eigenpairs, theta[nb] and C (k x nb, row-major) with C^T G C = I (all device FP64).  G is
 * scaled to unit diagonal and Cholesky-factored; *info_host (host int) = 0 on success, 1 when a
 * squared pivot fell below piv_tol (numerically dependent basis; C is then undefined). */
EIG_API eig_status eig_small_rr(const double* A, const double* G, int k, int nb, double piv_tol, double* theta,
                                double* C, int* info_host, void* stream);

/* 2x2 Rayleigh-Ritz of RMM-DIIS (Eqs. rr, xuwg) for m columns: dots (device FP64 m x 6 rows
 * <x,x>, <x,Hx>, <x,r>, <r,r>, <x,Hr>, <r,Hr>) -> theta[m] (smaller eigenvalue of the pencil)
 * and g[m][2] with g^T (W^T W) g = 1, g1 <= 0 (the orientation of LAPACK's generalized solver;
 * consecutive RMM-DIIS iterates alternate in sign).  active (device int[m]): 0 leaves the column on
 * x (g = (1/||x||, 0)). */
EIG_API eig_status eig_rmm_rr2(const double* dots, const int* active, int m, double* theta, double* g,
                               void* stream);

/* DIIS coefficients of Eqs. (xsum)-(rmm) for m columns: B (device FP64 [m][20][20]) holds the
 * residual Gram <r^(i), r^(k)> by history slot; slots (host int[s], oldest first, s <= 20)
 * name the window.  alpha (device FP64 [m][20]) receives the coefficients in window order
 * (sum 1), by the substitution alpha_last = 1 - sum(others) of Sec. 2.5 and a Cholesky solve
 * that drops the oldest entries while the difference system is numerically singular. */
EIG_API eig_status eig_rmm_diis(const double* B, const int* slots, int s, const int* active, int m, double* alpha,
                                void* stream);

/* ------------------------------------------------------------------------------------ *
 * Solver handle: eig_create / eig_solve / eig_ritz                                     *
 * ------------------------------------------------------------------------------------ */

typedef struct {
  double tol;              /* relative residual ||Hz - z theta|| / |theta| (Sec. 3.2); default 1e-6   */
  int maxiter;             /* iteration limit per phase; default 500                                */
  eig_method front;        /* hybrid front: EIG_LOBPCG (default) or EIG_BLOCK_LANCZOS (Sec. 4)      */
  double switch_tau;       /* hybrid: switch when tau (Eq. switchtau) <= switch_tau; default 1e-7;  */
                           /* <= 0 disables                                                          */
  double switch_res;       /* hybrid: switch when max rel. residual <= switch_res; default 0 (off)  */
  int switch_after;        /* hybrid: switch after this many front iterations; 0 = off              */
  int s_max;               /* DIIS window of Eqs. (xsum)-(rmm), 1..20; default 10 (Sec. 2.6)         */
  eig_dtype vec_type;      /* vector precision of the SpMM operands and front-phase blocks:         */
                           /* EIG_F32 (default, FP64 kept for Grams/projected problems/DIIS and the */
                           /* RMM-DIIS iterates) or EIG_F64 (every vector in FP64)                  */
  int precond;             /* LOBPCG K^{-1} of Eq. (wblock): 0 none, 1 Jacobi (default), 2 learned */
                           /* (eig_lp_*, parameters in lp_params)                                  */
  int rmm_precond;         /* RMM-DIIS: 0 W = (x~, r~) as Alg. 4 (default), 1 W = (x~, K^{-1} r~)  */
                           /* with Jacobi K, 2 with the learned K (FP32 vectors; FP64 vectors use  */
                           /* Jacobi)                                                               */
  double precond_floor;    /* Jacobi: |H_ii - theta| floored at this value; default 2.0 (two level  */
                           /* spacings of the CI spectrum: 0.1 amplifies near-degenerate rows)      */
  int cheb_degree;         /* ChebFSI polynomial degree d (Alg. 3); default 10 (Sec. 3.2)           */
  double lambda_ub;        /* ChebFSI spectrum upper bound; 0 = ten Lanczos steps (Sec. 3.2)        */
  int lanczos_maxbasis;    /* Lanczos / block Lanczos basis vectors before giving up; default 600   */
  const double* X0;        /* initial guess, FP64 row-major n x x0_cols, or NULL (seeded random)    */
  int x0_cols;
  int x0_on_device;
  uint64_t seed;           /* seed of the random start when X0 == NULL                              */
  int certify;             /* recompute true residuals in FP64 at the end (default 1)               */
  int timing;              /* record per-phase CUDA-event times in eig_stats (default 0)            */
  void* stream;            /* cudaStream_t; NULL = default stream                                   */
  double* trace;           /* optional host buffer of trace_cap rows of 2 + 2*n_ev doubles: per     */
  int trace_cap;           /* iteration [phase (0 front/single, 1 RMM-DIIS), iteration,             */
                           /* theta_1..theta_nev, relres_1..relres_nev] (the convergence histories  */
                           /* of Sec. 3.2); NULL = off                                              */
  int rmm_maxiter;         /* hybrid: RMM-DIIS iteration limit (0 = maxiter)                        */
  int rmm_fallback;        /* hybrid: when RMM-DIIS ends unconverged or with two collinear vectors, */
                           /* finish with LOBPCG on FP64 vectors from its result (default 1; 0 =   */
                           /* the paper's hybrid as printed, which has no remedy for that case)    */
  double diis_tol;         /* RMM-DIIS least squares: drop the oldest history entry while a squared */
                           /* Cholesky pivot of the normal matrix falls below diis_tol * its max   */
                           /* diagonal; 0 = by the residual history's precision (1e-6 for FP32,    */
                           /* 1e-13 for FP64)                                                       */
  const float* lp_params;  /* learned preconditioner (precond or rmm_precond = 2): host FP32 vector  */
                           /* of EIG_LP_PARAMS entries (layout at eig_lp_param_count); NULL = none */
  double switch_gap;       /* hybrid (not in the paper): switch only once, in addition to the rule   */
                           /* above, ||r_j|| <= switch_gap * gap_j for every wanted pair, gap_j the  */
                           /* distance from theta_j to the front's nearest other Ritz value: by     */
                           /* Davis-Kahan each Ritz vector is then within that angle of its          */
                           /* eigenvector, where RMM-DIIS (which converges to the eigenvector        */
                           /* nearest its start, Sec. 3.3) converges to the right one; 0 = off       */
                           /* (default).  Ignored with switch_after.                                 */
  int lanczos_keep;        /* block Lanczos thick restart (Sec. 2.2, restart after d iterations):   */
                           /* when the basis holds lanczos_maxbasis vectors (at most 62 blocks),    */
                           /* restart from the lowest lanczos_keep Ritz vectors (rounded up to a    */
                           /* multiple of the block, at least n_ev, at most 256 and one block below */
                           /* the basis) and the residual block; 0 (default) = half the basis;      */
                           /* -1 = no restart: stop at the basis limit                              */
  int rmm_decouple;        /* decoupled RMM-DIIS (Sec. 4.3): once this many wanted eigenvectors     */
                           /* have converged, each iteration forms H r~ by one SpMV per remaining   */
                           /* vector instead of one SpMM over the block (the same sums, so the same */
                           /* iterates); 0 (default) = coupled (SpMM) throughout.  Mirrored SpMM    */
                           /* layout only; other layouts stay coupled.                              */
} eig_opts;

typedef struct {
  int converged;           /* 1 when all n_ev pairs met tol                                          */
  int iterations_front;    /* front-method (or single-method) iterations                             */
  int iterations_rmm;      /* RMM-DIIS iterations (hybrid / rmmdiis)                                 */
  int switch_reason;       /* hybrid: 0 none, 1 tau, 2 residual, 3 fixed count, 4 front breakdown, */
                           /* 5 front residuals rising (instability)                               */
  int64_t spmm_calls;      /* products of H with a block                                            */
  int64_t spmv_count;      /* SpMV count as Sec. 2.6 counts it                                      */
  double last_tau;         /* last tau of Eq. (switchtau) seen by the front                          */
  double max_relres;       /* max relative residual of the returned pairs (FP64 if certify)         */
  double time_ms_total;    /* wall time of eig_solve on the stream (timing = 1)                     */
  double time_ms_spmm;     /* sum of SpMM kernel times (timing = 1)                                 */
  double time_ms_front;    /* front phase (timing = 1)                                              */
  double time_ms_rmm;      /* RMM-DIIS phase (timing = 1)                                           */
  int64_t spmm_timed;      /* SpMM calls included in time_ms_spmm                                   */
  double spmm_bytes;       /* sum over the solve's SpMM calls of their algorithmic bytes: one read  */
                           /* of the stored triangle (values + int32 columns) and rowptr, X read   */
                           /* and Y written once                                                     */
  int trace_rows;          /* rows written to opts->trace                                           */
  int iterations_fallback; /* LOBPCG iterations of the hybrid's fallback (0 when not needed)        */
  int precond_fallback;    /* learned preconditioner: 0 = used throughout; otherwise the (1-based)  */
                           /* iteration at which Jacobi replaced it (a step that raised the sum of */
                           /* the wanted Ritz values, or a non-finite m r): LOBPCG in the low 16   */
                           /* bits, RMM-DIIS in the high 16 bits                                    */
  int64_t lp_spmm_calls;   /* products H r spent on the learned preconditioner's features           */
  /* SpMM calls, CUDA-event time (timing = 1) and algorithmic bytes per product shape, index  */
  /* 6 * (vector type is EIG_F64) + log2(nb): e.g. 4 = FP32 vectors nb 16, 3 = FP32 nb 8,     */
  /* 9 = FP64 vectors nb 8                                                                     */
  int64_t spmm_calls_by_shape[12];
  double spmm_ms_by_shape[12];
  double spmm_bytes_by_shape[12];
  /* eig_solve_batch_ex with EIG_BATCH_LOCKSTEP: batched launches of the whole batch, and the  */
  /* products they carried (the same values in every instance's stats); 0 otherwise           */
  int64_t batch_launches;
  int64_t batch_products;
} eig_stats;

/* Fills *o with the defaults documented in eig_opts. */
EIG_API void eig_default_opts(eig_opts* o);

/* Creates a solver for the n_ev algebraically smallest eigenpairs of H (Sec. 2).  `block` is
 * the block size n_b >= n_ev of the block methods (Sec. 2.2-2.4; 8 or 16 in the paper); it is
 * rounded up to a power of two <= 32.  H is copied to device memory owned by the handle and the
 * SpMM plan is built (see eig_spmm_plan_create).  One handle serves one stream at a time.
 * Errors: EIG_EINVAL (n_ev < 1, n_ev > block, block > 32, n_ev > n, malformed CSR). */
EIG_API eig_status eig_create(const eig_csr_upper* H, int n_ev, int block, void** handle);
/* eig_create with the SpMM plan's device layout chosen explicitly (an eig_layout). */
EIG_API eig_status eig_create_ex(const eig_csr_upper* H, int n_ev, int block, int layout, void** handle);
/* Description of the SpMM plan a solver handle built (layout, tiles, device bytes). */
EIG_API eig_status eig_solver_spmm_info(const void* handle, eig_spmm_info* info);
EIG_API void eig_destroy(void* handle);

/* Runs a method (opts NULL = defaults).  Returns EIG_OK when every pair met opts->tol,
 * EIG_ENOT_CONVERGED when maxiter ran out (the best pairs are still kept for eig_ritz),
 * EIG_EBREAKDOWN when a basis became numerically rank deficient before any usable result,
 * EIG_EDUPLICATE when RMM-DIIS left two returned vectors on the same eigenvector.
 * stats may be NULL.  Synchronises opts->stream before returning. */
EIG_API eig_status eig_solve(void* handle, eig_method method, const eig_opts* opts, eig_stats* stats);

/* Copies the last result: theta[n_ev] (host, ascending), X (FP64 row-major n x n_ev, host when
 * on_device = 0, device otherwise; may be NULL), relres[n_ev] (host; may be NULL).
 * EIG_EINVAL when no solve has produced a result yet. */
EIG_API eig_status eig_ritz(void* handle, double* theta, double* X, double* relres, int on_device);

/* ------------------------------------------------------------------------------------ *
 * Batches of independent instances and the SpMM plan autotuner                         *
 * ------------------------------------------------------------------------------------ *
 * Secs. 1 and 4.3 argue for concurrency at the level of eigenpairs: independent small pieces of
 * work only fill a wide machine when they run side by side.  Many small matrices (each far too
 * small to fill 152 SMs, each synchronising with the host once per iteration) are solved
 * together by eig_solve_batch. */

/* eig_create_ex with the SpMM plan's row block R and column block C given (0 = 256 / 64; see
 * eig_spmm_plan_create_ex for the constraints), e.g. the shape eig_autotune_spmm chose. */
EIG_API eig_status eig_create_ex2(const eig_csr_upper* H, int n_ev, int block, int layout, int row_block,
                                  int col_block, void** handle);

/* eig_create_ex for count matrices Hs[0..count) with one n_ev, block and layout: handles[i]
 * (caller array of count pointers).  All or nothing: on an error every handle already created
 * is destroyed, all entries are NULL, and the first error is returned. */
EIG_API eig_status eig_create_batch(const eig_csr_upper* Hs, int count, int n_ev, int block, int layout,
                                    void** handles);

/* Solves count independent instances (handles from eig_create*) with one method.  opts: NULL =
 * defaults for all; otherwise opts[i] for instance i when per_instance_opts != 0, else opts[0]
 * for all (an X0 given there is then shared).  `threads` host threads (0 = min(count, 16)) take
 * instances in index order; each owns a non-blocking stream, used by every instance whose
 * opts.stream is NULL, so the instances' kernels overlap on the GPU.  The results are those of
 * eig_solve on each handle alone (every kernel is deterministic).  status[i], stats[i] (may be
 * NULL) receive each instance's eig_solve result.  Returns EIG_OK, or the first status other
 * than EIG_OK / EIG_ENOT_CONVERGED / EIG_EDUPLICATE.  A handle must not appear twice. */
EIG_API eig_status eig_solve_batch(void* const* handles, int count, eig_method method, const eig_opts* opts,
                                   int per_instance_opts, int threads, eig_status* status, eig_stats* stats);

/* Flags of eig_solve_batch_ex. */
#define EIG_BATCH_LOCKSTEP 1

/* eig_solve_batch with flags.  EIG_BATCH_LOCKSTEP: the products of the running instances are
 * launched together -- each instance's next SpMM (or fused Chebyshev step) waits until every
 * running instance has posted its own, then one launch per product shape covers all of them,
 * its CTAs the concatenated row blocks of the posted products (the (instance, row block) work
 * list); an instance that has finished leaves the rounds (per-instance convergence).  Every
 * other step of a solve still runs on its instance's stream.  Batched shapes: mirrored plans,
 * FP32 values, block 8 or 16, FP32 or FP64 (double-float) vectors; other products of a round
 * are launched one by one.  The results are bitwise those of eig_solve on each handle alone
 * (each product sums in the single launch's order).  stats[i].batch_launches / batch_products
 * count the batched launches and the products they carried. */
EIG_API eig_status eig_solve_batch_ex(void* const* handles, int count, eig_method method, const eig_opts* opts,
                                      int per_instance_opts, int threads, int flags, eig_status* status,
                                      eig_stats* stats);

typedef struct {
  int layout;       /* eig_layout */
  int row_block;    /* R */
  int col_block;    /* C */
  double ms;        /* mean time of one SpMM with the tuning block */
} eig_tune_result;

/* Times Y = H X (nb columns of vec_type, reps repetitions after two warm-ups) for each
 * candidate plan shape -- mirrored (256/64), half-stored tiles (256/64, 128/64, 512/128), CSR
 * (256/64, 128/32, 512/64) -- and returns the fastest in *best; all[] (room for 8, may be NULL)
 * and *n_all receive every shape that could be built.  H on host or device (copied once).
 * Synchronises stream.  EIG_EUNSUPPORTED when no shape could be built. */
EIG_API eig_status eig_autotune_spmm(const eig_csr_upper* H, int nb, eig_dtype vec_type, int reps,
                                     eig_tune_result* best, eig_tune_result* all, int* n_all, void* stream);

/* The Chebyshev degree d of Alg. 3 for this handle's matrix: after one untimed warm-up solve,
 * runs the ChebFSI solve (opts from base, NULL = defaults; cheb_degree and timing overridden)
 * three times per degrees[i] and returns in *best_degree the degree with the smallest median
 * time_ms_total among those whose runs all converged; ms[i] (the median, 0 when not a
 * candidate) and converged[i] (may be NULL) receive each degree's result.  A degree whose
 * solve does not converge, returns duplicate pairs or breaks down is skipped, not fatal.  The
 * handle keeps the result of the last run.  EIG_ENOT_CONVERGED (and *best_degree = 0) when no
 * degree converged; CUDA, allocation and argument errors are returned at once.
 * Synchronises base->stream. */
EIG_API eig_status eig_autotune_cheb(void* handle, const int* degrees, int count, const eig_opts* base,
                                     int* best_degree, double* ms, int* converged);

/* ------------------------------------------------------------------------------------ *
 * Learned per-row preconditioner (a replacement for K of Eq. (wblock))                 *
 * ------------------------------------------------------------------------------------ *
 * The paper leaves K open: it only has to approximate H (Sec. 2.3), and Secs. 5-6 name a
 * better preconditioner as the way to cut iterations further.  The learned K^{-1} scales each
 * residual entry, w_ij = m_ij r_ij, by m_ij = J_ij (1 + o_ij): J_ij = 1 / floor(H_ii - theta_j) is
 * the Jacobi scale (|.| floored at 2, sign kept) and o_ij = MLP(f_ij) a learned correction, so a
 * zero output layer is exactly the Jacobi K.  Six features of row i and column j:
 *   f0 = H_ii, f1 = theta_j, f2 = H_ii - theta_j, f3 = (|H| 1)_i (absolute row sum of the full H),
 *   f4 = sqrt(n) r_ij / ||r_j||, f5 = sqrt(n) ((H - D) r_j)_i / ||r_j||  (0 for a zero column).
 * Network 6 -> 32 -> 32 -> 1, ReLU after both hidden layers, FP32, on u = (f - mu) / sigma.
 * Parameter vector (FP32, EIG_LP_PARAMS entries, in this order):
 *   mu[6] sigma[6] W1[32][6] b1[32] W2[32][32] b2[32] w3[32] b3
 * mu and sigma are fixed feature statistics; the EIG_LP_TRAINED entries after them are trained.
 * Where m r is not finite the entry takes the Jacobi value r / floor(H_ii - theta_j).
 * Training target: the Jacobi-Davidson correction to first order measured against the
 * converged wanted space X* (orthonormal n x k): z_j = x_j - X* p / (p^T p), p = X*^T x_j; loss
 * L = (1/|J|) sum_{j in J} sum_i (m_ij r_ij - z_ij)^2 / ||z_j||^2 over the columns J with a
 * target. */
#define EIG_LP_PARAMS 1325
#define EIG_LP_TRAINED 1313

/* Number of entries of a parameter vector (EIG_LP_PARAMS). */
EIG_API int eig_lp_param_count(void);

/* One training sample from the solver's matrix.  X (device FP64 n x m row-major, m <= 32) and
 * theta (host FP64 [m]) are Ritz pairs of H; the call forms R = H X - X diag(theta) and H R with
 * the handle's SpMM plan and writes, all on the device:
 *   F[(i*m + j)*6 + q] (FP32 features), r[i*m + j] (FP32 residual), z[i*m + j] (FP32 target),
 *   colw[j] (FP64 weight of column j in the loss: 1 / (|J| ||z_j||^2), or 0 without a target).
 * target 0: the correction target against Xstar (device FP64 n x k row-major, 1 <= k <= 32,
 * orthonormal); target 1: the Jacobi target z = r / floor(H_ii - theta_j) (Xstar unused),
 * used to start a network from Jacobi.  floor: the Jacobi floor (eig_opts.precond_floor).
 * Synchronises stream.  Errors: EIG_EINVAL (sizes, null pointers). */
EIG_API eig_status eig_lp_sample(void* handle, const double* X, int m, const double* theta, const double* Xstar,
                                 int k, int target, double floor, float* F, float* r, float* z, double* colw,
                                 void* stream);

/* W = K^{-1} R with the learned K (params: host FP32 vector).  R, W: device n x m row-major of
 * vec_type (EIG_F32 or EIG_F64), m a power of two <= 32, W may equal R; theta host FP64 [m].
 * One SpMM of R with the handle's plan forms f5.  Synchronises stream. */
EIG_API eig_status eig_lp_apply(void* handle, const float* params, const void* R, int m, eig_dtype vec_type,
                                const double* theta, double floor, void* W, void* stream);

/* m_out[e] = MLP(F[e*6 .. e*6+5]) for e < count (device FP32 in and out; params host FP32). */
EIG_API eig_status eig_lp_forward(const float* params, const float* F, int64_t count, float* m_out, void* stream);

/* Device scratch bytes eig_lp_grad needs. */
EIG_API size_t eig_lp_grad_workspace_bytes(void);

/* Loss and gradient of one sample (F, r, z, colw from eig_lp_sample; n rows, m columns):
 * grad (device FP64 [EIG_LP_TRAINED + 1]) receives dL/d(params[12 + q]) for q < EIG_LP_TRAINED,
 * then L.  params: device FP32 vector.  Deterministic (fixed-order reductions). */
EIG_API eig_status eig_lp_grad(const float* params, const float* F, const float* r, const float* z,
                               const double* colw, int64_t n, int m, double* grad, void* workspace, void* stream);

/* One Adam step (Kingma & Ba) on the trained entries of params (device FP32) from grad
 * (eig_lp_grad); m1, m2: device FP32 moment vectors of EIG_LP_PARAMS entries (start at zero);
 * t: 1-based step count of the bias corrections. */
EIG_API eig_status eig_lp_adam(float* params, const double* grad, float* m1, float* m2, int t, double lr,
                               double beta1, double beta2, double eps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* EIG_H_ */
