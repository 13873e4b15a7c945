/*
 * rks.h - C ABI of librks: randomized Krylov-Schur (rKS) with deflation on a
 * GB300 GPU (sm_103a).
 *
 * The solver computes k eigenpairs (lambda, x) of a sparse non-symmetric
 * A in R^{n x n} (CSR), A x = lambda x (Eq. 2.1), following Algorithm 1 (rKS)
 * and Algorithm 2 (extension by randomized Arnoldi) of de Damas & Grigori,
 * "Randomized Krylov-Schur eigensolver with deflation", with the locking of
 * converged Schur vectors of Sec. 4.2-4.4 and the residual estimates of
 * Sec. 4.1.  The Krylov dimension is m = k + p; Omega in R^{d x n} is a
 * sparse-sign embedding (zeta nonzeros +-1/sqrt(zeta) per column, rows and
 * signs from a SplitMix64 hash of (seed, column), see rks_sketch_pairs).
 *
 * Conventions for every entry point:
 *  - return value: RKS_OK (0) or a negative rks_status; no exceptions cross
 *    the ABI; rks_strerror() gives a static message;
 *  - dense arrays are column-major; "n x k" means n rows;
 *  - array arguments are host pointers unless opts.mem_device = 1 was given
 *    to rks_create, in which case the arrays passed to rks_create,
 *    rks_get_schur and rks_get_eigpairs (not rks_info) are device pointers
 *    of the current CUDA device;
 *  - the caller owns every array it passes; rks_create copies A (and u1)
 *    into memory owned by the context; rks_destroy frees it all;
 *  - a context is used by one host thread at a time; its kernels run on
 *    opts.stream (a cudaStream_t), or on a stream the context creates.
 */
#ifndef RKS_H
#define RKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rks_ctx rks_ctx;

typedef enum {
  RKS_OK = 0,
  RKS_EINVAL = -1,      /* invalid argument (sizes, CSR structure, d < 2*zeta, ...) */
  RKS_ENOMEM = -2,      /* device or host allocation failed */
  RKS_ECUDA = -3,       /* a CUDA call failed */
  RKS_ENOCONV = -4,     /* maxit restarts without convergence: results are the
                           current (partial) decomposition and are valid */
  RKS_EBREAKDOWN = -5,  /* beta_{j+1} = 0: an invariant subspace was reached
                           before k pairs converged (Sec. 2.1) */
  RKS_ENAN = -6,        /* a non-finite value appeared (e.g. NaN in A) */
  RKS_ESTATE = -7,      /* call out of order (e.g. rks_get_* before rks_solve) */
  RKS_EDENSE = -8,      /* the small dense Schur iteration failed */
  RKS_ETIMEOUT = -9     /* a bounded device-side wait (grid barrier) timed out */
} rks_status;

/* Wanted part of the spectrum (Sec. 5: largest / smallest modulus; real part). */
typedef enum { RKS_LM = 0, RKS_SM = 1, RKS_LR = 2, RKS_SR = 3 } rks_which;

/* Element type of the CSR values passed to rks_create. */
typedef enum { RKS_F64 = 0, RKS_F32 = 1 } rks_dtype;

typedef struct {
  int zeta;            /* nonzeros per column of Omega; default 8 */
  int maxit;           /* maximum number of restarts; default 1000 */
  int lock;            /* 1: lock converged Schur vectors (Sec. 4.4); default 1 */
  int mem_device;      /* 1: array arguments are device pointers; default 0 */
  void* stream;        /* cudaStream_t for all work; NULL: the context's own */
  const double* u1;    /* start vector (n), host or device per mem_device;
                          NULL: N(0,1) entries from SplitMix64(seed + 1) and
                          Box-Muller, generated on the device */
  double eta_lock;     /* locking threshold, relative to |lambda|; 0: tol */
  int max_restarts;    /* stop after this many contractions whatever the
                          estimates say (fixed-iteration runs, Sec. 5); 0: none;
                          -1: only the initial expansion of Algorithm 1 */
  int profile;         /* 1: time every kernel launch with CUDA events on the
                          context's stream (see rks_get_stats); default 0.
                          profile > 1: time only the launches of the kernel
                          classes whose bits are set in profile >> 1 (bit c
                          for class c of RKS_K_*), e.g.
                          1 | 2 << RKS_K_UPDATE for the update kernel alone:
                          fewer events in the stream */
  int conv;            /* convergence scale, RKS_CONV_EIG (default) or
                          RKS_CONV_NORM1, see below */
  int prec;            /* arithmetic of the n-dimensional work:
                          RKS_PREC_DF (default): basis and matrix values stored
                          as float pairs (hi + lo, 48-bit significand, 8 bytes),
                          products and sums by error-free transformations on the
                          FP32 pipes; RKS_PREC_FP64: native FP64;
                          RKS_PREC_MIXED: FP32 basis and FP32 matrix values with
                          compensated (error-free) products and sums until
                          the estimates reach mixed_tol or stagnate.  With
                          keep > 0 this phase does not lock and the
                          double-float restarts continue from its
                          Krylov-Schur decomposition A U = U T + u b^T: U
                          promoted exactly,
                          its relation error (the FP32 rounding of the stored
                          vectors) reduced by damped Jacobi sweeps on
                          A X - X T = -(A U - U T - u b^T) with U <- U + X,
                          [U u] re-orthonormalised in the sketch.  With
                          keep = 0, or if the relation error left is above
                          what tol asks (see rks_stats.handover_rel) or that
                          phase stagnates, a double-float solve started from
                          the sum of the FP32 Schur vectors finishes to tol.
                          The sketch sums, the small dense work and the final
                          residuals are FP64 in all three. */
  double mixed_tol;    /* RKS_PREC_MIXED: tolerance of the FP32 phase on the
                          opts.conv scale; 0: 32 * 2^-24 with keep > 0, 64 * 2^-24 with keep = 0 */
  double verify;       /* > 0: after convergence, check the FP64 residuals
                          ||A x - l x|| / (||A||_1 ||x||) <= verify; if one
                          fails, divide tol and eta_lock by 4 and continue the
                          restarts from the current decomposition (bounded
                          by maxit); 0: no check (default) */
  int keep;            /* 0 (default): a restart keeps the k - q best active
                          Schur vectors (Algorithm 1 truncates to k, q locked).
                          1..k: thick restart, it keeps
                          max(k - q, min(keep, (m - q) / 2)) of them, so that
                          after locking the restart still carries up to keep
                          active directions.  Either way convergence and the
                          reported Ritz pairs concern the rks_nwanted best
                          Ritz pairs of the kept decomposition. */
  int ortho;           /* RKS_ORTHO_SKETCH (default): randomized Gram-Schmidt
                          in the sketch (the method).  RKS_ORTHO_CGS2: the
                          Krylov-Schur baseline the paper compares against
                          (KS-CGS2, Sec. 5): Euclidean classical Gram-Schmidt
                          with reorthogonalisation, same storage and kernels,
                          no sketch; RKS_PREC_DF only. */
  int tc_restart;      /* 1 (default): the restart product U_k = U Q' (Eq. 3.5)
                          runs on the tensor cores where its sizes allow
                          (at most 64 output columns, 256 input columns for
                          the FP32 basis and 192 for the double-float basis,
                          and the digit image of Q' in shared memory):
                          split-BF16 products for the FP32 basis, exact 7-bit
                          digit products (FP64-class) for the double-float
                          basis;
                          0: the SIMT kernels. */
  int aggressive;      /* 1: aggressive deflation (Sec. 4.3, after Thm 4.3):
                          before locking, the active Schur form is reordered
                          (orthogonal swaps of diagonal blocks) so that every
                          block whose Ritz estimate |b^T y| is below the
                          locking threshold leads, converged blocks in their
                          order, then the others in theirs; the leading ones
                          then lock as usual.  Needs lock = 1.  Nothing moves
                          if a swap is refused.  0 (default): only a leading
                          prefix of converged Schur vectors locks. */
  int debug_stall;     /* test hook for the failure path: 1 makes every grid
                          barrier of the cooperative least-squares kernel wait
                          for one CTA more than the grid holds, so each wait
                          runs out its short limit (about a millisecond), the
                          kernel records the timeout and finishes, and
                          rks_solve returns RKS_ETIMEOUT; the context's
                          barrier state is reset and the device stays usable.
                          0 (default): off. */
} rks_opts;

enum { RKS_ORTHO_SKETCH = 0, RKS_ORTHO_CGS2 = 1 };

enum { RKS_PREC_DF = 0, RKS_PREC_FP64 = 1, RKS_PREC_MIXED = 2 };

/* Convergence test on the Ritz pairs (lambda_i, y_i) of T, ||y_i|| = 1:
 *  RKS_CONV_EIG   |b^T y_i| / |lambda_i| <= tol   (Eq. 4.8, Sec. 5.1), and
 *                 locking when |b_i| <= eta_lock * |lambda_i|;
 *  RKS_CONV_NORM1 |b^T y_i| / ||A||_1 <= tol      (the non-relative bound of
 *                 the Sec. 4.1 remark, ||Ax - lx|| / ||x|| ~ |b^T y|, scaled
 *                 by ||A||_1), and locking when |b_i| <= eta_lock * ||A||_1
 *                 (the absolute threshold of Eq. 4.21 with eta = eta_lock ||A||_1). */
enum { RKS_CONV_EIG = 0, RKS_CONV_NORM1 = 1 };

typedef struct {
  int nconv;           /* number of pairs whose estimate is <= tol */
  int nlocked;         /* locked Schur vectors q */
  int restarts;        /* contractions performed */
  int64_t nmatvec;     /* products with A */
  int converged;       /* 1 if all k estimates are <= tol */
  double max_est;      /* max_i |b^T y_i| / |lambda_i| (Eq. 4.8) */
  double max_resid;    /* max_i ||A x_i - lambda_i x_i|| / (||A||_1 ||x_i||), FP64 */
  double t_solve_ms;   /* wall time of rks_solve (CUDA events on the stream) */
} rks_info;

/* Kernel classes of rks_stats: the steps of one Arnoldi step of Algorithm 2
 * and of the restart of Algorithm 1. */
enum {
  RKS_K_SPMV = 0,      /* w = A u_j fused with z = Omega w */
  RKS_K_LS = 1,        /* b = S^+ z (CGS2 in the sketch), three small kernels */
  RKS_K_UPDATE = 2,    /* u~ = w - U b fused with s~ = Omega u~ */
  RKS_K_FINISH = 3,    /* beta = ||s~||, append to S and B */
  RKS_K_RESTART = 4,   /* U_k = U Q (Eq. 3.5) */
  RKS_K_OTHER = 5,     /* start vector, Ritz vectors, residuals */
  RKS_NK = 6
};

/* Counters of the last rks_solve.  launches counts every kernel the library
 * launched.  ms (event time) is filled for the timed classes when
 * opts.profile is set, else 0.  bytes
 * and flops are the algorithmic traffic / work of the launches: SpMV
 * nnz*(P_A + 4) + 4(n+1) + 2 P_V n; update (c + 2) P_V n for c basis
 * columns; restart (m_a + k_a + 2) P_V n; P = bytes per value. */
typedef struct {
  int64_t launches[RKS_NK];
  double ms[RKS_NK];
  double bytes[RKS_NK];
  double flops[RKS_NK];
  double host_ms;      /* host time in the small dense step (Schur ... locking) */
  int64_t whitenings;  /* restarts that whitened the kept sketches (Sec. 3.3) */
  int64_t reorders;    /* restarts whose aggressive deflation moved a block */
  int fp32_restarts;   /* RKS_PREC_MIXED: restarts of the FP32 phase */
  int mixed_phase2;    /* RKS_PREC_MIXED: how the double-float phase began:
                          0 none (the FP32 result met the target), 1 from the
                          FP32 decomposition made exact (see opts.prec),
                          2 from the sum of the FP32 Schur vectors */
  double handover_rel; /* RKS_PREC_MIXED: largest column norm of the relation
                          error A U - U T - u b^T left by the correction, over
                          ||A||_1 (phase 2 continues from it only when it is
                          below what the target asks: tol on the ||A||_1
                          scale, verify - tol with the FP64 check, tol times
                          the smallest wanted |lambda| / ||A||_1 on the
                          |lambda| scale; otherwise mixed_phase2 = 2) */
  int64_t launches_f32[RKS_NK];   /* the part of launches, ms and bytes above */
  double ms_f32[RKS_NK];          /* made with the FP32 basis (RKS_PREC_MIXED's */
  double bytes_f32[RKS_NK];       /* first phase) */
} rks_stats;

/* Counters of the last rks_solve (see rks_stats). */
int rks_get_stats(const rks_ctx* c, rks_stats* out);

/* Fill *o with the defaults above. */
void rks_opts_default(rks_opts* o);

/* Create a solver for A (n x n, CSR: rowptr[n+1], colind[nnz] (0-based, each
 * row's columns in [0, n)), vals[nnz] of type vals_dtype).  k wanted pairs,
 * p extra Krylov directions (m = k + p, 1 <= k, 2 <= p, m + 1 <= n), sketch
 * size d (d >= m + 1 and d >= 2*zeta), which part of the spectrum, tolerance
 * tol > 0 on the estimates |b^T y|/|lambda| (Sec. 5.1), and the seed of
 * Omega.  opts may be NULL (defaults).  Copies A to the device and validates
 * its structure (rowptr non-decreasing, rowptr[0] = 0, column indices in
 * range); on error *out is NULL. */
int rks_create(rks_ctx** out, int64_t n, const int32_t* rowptr, const int32_t* colind,
               const void* vals, int vals_dtype, int k, int p, int d, int which,
               double tol, uint64_t seed, const rks_opts* opts);

/* Run Algorithm 1 to convergence (or maxit / max_restarts).  info may be
 * NULL.  Returns RKS_OK, RKS_ENOCONV (results valid but not converged),
 * RKS_EBREAKDOWN, RKS_ENAN or a CUDA error.  May be called again: it
 * restarts from the start vector. */
int rks_solve(rks_ctx* c, rks_info* info);

/* The rKS decomposition A U = U T + u b^T of the last solve (Def. 2.9), with
 * kk = rks_nkept(c) columns: the q locked and the active Schur vectors kept
 * at the last restart (k, or k + 1 when a complex pair straddles the cut; up
 * to q + keep with opts.keep > 0).  T: kk x kk (host, FP64); U: n x kk FP64
 * (host or device per mem_device), unit sketch norm columns
 * ||Omega U e_i|| = 1; b: kk (host).  Any pointer may be NULL. */
int rks_get_schur(rks_ctx* c, double* T, double* U, double* b);

/* Storage the SpMV of a context reads, chosen at rks_create from the
 * structure of A (double-float and mixed paths; the FP64 path reads CSR):
 *   RKS_SPMV_CSR    CSR, two rows per thread (short, even rows);
 *   RKS_SPMV_ELL    ELLPACK interleaved by 32-row slices (rows of at most 16
 *                   entries with little padding);
 *   RKS_SPMV_DIA    by diagonals (at most 16 distinct column - row offsets,
 *                   little padding: stencils);
 *   RKS_SPMV_WARP   CSR, one warp per row (mean row length >= 16);
 *   RKS_SPMV_MERGE  CSR by merge path: rows + entries split evenly over the
 *                   threads, partial rows folded in thread order, then the
 *                   sketch (longest row > 128 and > 16 x the mean).
 * The sum of a row is in column order for CSR, ELL and DIA (the same bits),
 * lane-strided for WARP and split at thread boundaries for MERGE; every
 * variant is deterministic.  Returns the format or RKS_EINVAL. */
enum { RKS_SPMV_CSR = 0, RKS_SPMV_ELL = 1, RKS_SPMV_DIA = 2, RKS_SPMV_WARP = 3, RKS_SPMV_MERGE = 4 };
int rks_spmv_format(const rks_ctx* c);

/* Number of columns kk of the decomposition returned by rks_get_schur. */
int rks_nkept(const rks_ctx* c);

/* Number nw of Ritz pairs reported by rks_get_eigpairs and
 * rks_get_estimates: the best k of the kept decomposition, k + 1 when the
 * k-th is the first member of a complex pair (at most kk). */
int rks_nwanted(const rks_ctx* c);

/* Ritz pairs of the last solve, best first (Sec. 4.1): lam_re, lam_im (nw,
 * host); X (n x nw FP64, host or device per mem_device) in LAPACK dgeev real
 * packing: a conjugate pair occupies columns (j, j+1) = (Re x, Im x) of the
 * eigenvector of the member with Im > 0; resid (nw, host) =
 * ||A x - lambda x|| / (||A||_1 ||x||) computed in FP64 on the device.  Any
 * pointer may be NULL. */
int rks_get_eigpairs(rks_ctx* c, double* lam_re, double* lam_im, double* X, double* resid);

/* Rayleigh quotients lambda_RQ,i = x_i^H A x_i / x_i^H x_i of the Ritz
 * vectors x_i = U Y e_i returned by rks_get_eigpairs (the refined eigenvalue
 * estimate that goes with the residual of Sec. 4.1), in the same order, nw
 * values each (host).  x^H A x and x^H x are summed in FP64 on the device
 * from the FP64 Ritz vector and the FP64 product A x (the pass that gives the
 * residuals), per-CTA partial sums added on the host in CTA order.  For a
 * conjugate pair the member with Im > 0 gets x^H A x / x^H x of its complex
 * eigenvector and its partner the conjugate.  Either pointer may be NULL.
 * Returns RKS_OK, RKS_EINVAL or RKS_ESTATE (no completed solve). */
int rks_get_rayleigh(rks_ctx* c, double* rq_re, double* rq_im);

/* Residual estimates |b^T y_i| / |lambda_i| (Eq. 4.8) of the last solve, in
 * the order of rks_get_eigpairs (nw values, host). */
int rks_get_estimates(rks_ctx* c, double* est);

/* The sketch-orthonormal Krylov decomposition as it stands (for tests of
 * Algorithm 2): ncols_out = number of basis columns j + 1 (locked + active
 * + the last vector u).  U: n x (j+1) FP64 with unit sketch norm columns,
 * S = Omega U: d x (j+1), H: (j+1) x j with column i holding the projection
 * coefficients of A u_i on u_0..u_i (rows 0..i) and beta_{i+1} (row i+1),
 * for the columns produced by the last expansion (other entries 0).
 * Array pointers may be NULL; sizes must allow m + 1 columns.  Host
 * pointers only. */
int rks_get_krylov(rks_ctx* c, int* ncols_out, double* U, double* S, double* H);

/* Convergence history of the last rks_solve: after restart i, hist[i] =
 * max over the Ritz pairs of the convergence quantity of opts.conv and
 * nlock[i] = locked vectors.  Writes min(cap, restarts) entries and returns
 * their number (negative on error).  Either pointer may be NULL. */
int rks_get_history(const rks_ctx* c, double* hist, int* nlock, int cap);

/* ||A||_1 (max column sum of |a_ij|), computed at rks_create. */
double rks_norm1(const rks_ctx* c);

/* Free everything owned by the context (device memory, stream, events).
 * Safe on NULL. */
void rks_destroy(rks_ctx* c);

/* Static message for a status code. */
const char* rks_strerror(int status);

/* ---- Batched solve of independent problems --------------------------- */

/* Many independent problems (e.g. a batch of uneven operators) solved
 * concurrently: one context per problem, each on a stream of its own, up to
 * nthreads problems in flight with their small dense steps on separate host
 * threads.  The kernels are deterministic, so every problem's results are the
 * bits of a solve of that problem alone. */
typedef struct rks_batch rks_batch;

/* One context per problem i < count from its CSR arrays (rowptr[i], colind[i],
 * vals[i]; host or device pointers per opts.mem_device) and n[i]; every other
 * argument is shared and means what it means for rks_create.  opts.stream and
 * opts.u1 must be NULL (each context creates its stream and draws its start
 * vector from seed + 1).  Contexts are created on up to nthreads host threads.
 * On failure nothing is kept and the first failing status in problem order is
 * returned. */
int rks_create_batched(rks_batch** out, int count, const int64_t* n, const int32_t* const* rowptr,
                       const int32_t* const* colind, const void* const* vals, int vals_dtype, int k, int p,
                       int d, int which, double tol, uint64_t seed, const rks_opts* opts, int nthreads);

/* rks_solve of every problem, up to nthreads at a time; infos (count entries,
 * may be NULL) receives each problem's rks_info.  Returns RKS_OK, RKS_ENOCONV
 * when some problem did not converge (its results are partial) and no other
 * error occurred, else the first other failing status in problem order;
 * rks_batch_status gives each problem's own status. */
int rks_solve_batched(rks_batch* b, int nthreads, rks_info* infos);

/* Number of problems; the context of problem i (borrowed: valid until
 * rks_destroy_batched, for rks_get_eigpairs and the other getters; NULL if i
 * is out of range); the status of its last create or solve. */
int rks_batch_count(const rks_batch* b);
rks_ctx* rks_batch_get(rks_batch* b, int i);
int rks_batch_status(const rks_batch* b, int i);

/* Free every context of the batch.  Safe on NULL. */
void rks_destroy_batched(rks_batch* b);

/* ---- Batched solve in one persistent launch -------------------------- */

/* Many independent problems solved by persistent kernels (Algorithm 1 with
 * Algorithm 2 for every problem, the small dense steps on the device) in one
 * CUDA graph: clusters of G CTAs (G = 1, 2, 4 or 8) take problems from a
 * device work queue sorted by cost (nnz + n m), largest first; the rows of a
 * problem are split over the CTAs of its cluster.  A configuration is one
 * kernel, or two running at once: clusters of GL CTAs taking problems from the
 * front of the queue and clusters of GS < GL CTAs taking them from the back
 * (one atomic counter pair, so the two ends never take the same problem).  Double-float basis and matrix values,
 * FP64 sketch sums, least squares, dense steps and residuals; the restart
 * keeps the max(k, min(opts.keep, m / 2)) best Schur vectors (a thick restart;
 * the truncation of Algorithm 1 with a larger size) and locks nothing;
 * convergence when the rks_nwanted best estimates (opts.conv scale) are <= tol,
 * then, if opts.verify > 0, the FP64 residuals ||A x - l x|| / (||A||_1 ||x||)
 * must be <= verify, else tol is divided by 4 and the restarts go on (bounded
 * by opts.maxit).  Omega is the sparse-sign embedding of rks_create for every
 * problem (rks_sketch_pairs with `seed`), the start vector the default of
 * rks_create (SplitMix64(seed + 1)).  Every reduction has a fixed order that
 * does not depend on G or on the other problems: a problem's results are the
 * same bits in any batch and for any G. */
typedef struct rks_dbatch rks_dbatch;

/* Problems i < count from host CSR arrays (rowptr[i], colind[i], vals[i] of
 * vals_dtype, n[i] rows; values finite and |v| <= 3e38); k, p (m = k + p <= 64,
 * k + 1 <= 32, p >= 2), d (>= m + 1, >= 2 zeta), which, tol and seed as for
 * rks_create; max(k, min(opts.keep, m / 2)) + 1 <= 32.  Of opts (may be
 * NULL) zeta, maxit, conv, verify, keep and stream are used; mem_device and u1
 * must be 0 / NULL; the other fields are ignored.
 * ctas_per_problem: 1, 2, 4 or 8 CTAs per problem (one kernel), or 0 to time
 * candidate configurations (one kernel with G = 2, 4, 8; two kernels with
 * (GL, GS) = (8, 2), (8, 4), (4, 2) sharing the CTA slots) on a tuning run of
 * two restarts of every problem, and keep the fastest (rks_dbatch_config).
 * Copies everything to the device (the caller keeps its arrays) and captures
 * the launch in a CUDA graph.  RKS_EINVAL for an invalid argument or a
 * problem whose shared-memory layout exceeds the device's limit. */
int rks_create_batched_dev(rks_dbatch** out, int count, const int64_t* n, const int32_t* const* rowptr,
                           const int32_t* const* colind, const void* const* vals, int vals_dtype, int k, int p,
                           int d, int which, double tol, uint64_t seed, const rks_opts* opts, int ctas_per_problem);

/* One launch of the captured graph for all problems; infos (count entries,
 * may be NULL) receive restarts, nmatvec, converged, nconv, max_est,
 * max_resid (nlocked = 0) and t_solve_ms (the launch's event time, the same
 * for every problem).  Returns the first status other than RKS_OK and
 * RKS_ENOCONV in problem order, else RKS_ENOCONV if a problem did not
 * converge, else RKS_OK. */
int rks_solve_batched_dev(rks_dbatch* b, rks_info* infos);

/* The launch configuration: cfg4 = {GL, nL, GS, nS} (nL clusters of GL CTAs
 * from the front of the queue, nS clusters of GS CTAs from the back; nS = 0
 * for one kernel), the times (ms) of the first ntune tuning runs in candidate
 * order, and the event time of the last solve; returns the number of tuning
 * runs (1 when the configuration was given).  Any pointer may be NULL. */
int rks_dbatch_config(const rks_dbatch* b, int* cfg4, float* tune_ms, int ntune, float* last_ms);

/* Status of problem i in the last solve (RKS_ESTATE before one). */
int rks_dbatch_status(const rks_dbatch* b, int i);

/* Cycle counts of the last solve by phase, summed over CTAs and problems
 * (clock64 deltas taken by thread 0 of every CTA at the barriers that end
 * each phase): 0 start vector, 1 SpMV rows with the sketch sums of w, 2
 * Hessenberg reduction, 3 exchanges of the sketch sums, 4 least squares, 5
 * update rows with the sketch sums of u~, 6 Francis QR iteration, 7 beta and
 * append, 8 reordering and truncation, 9 kept sketches and
 * whitening, 10 restart product, 11 Ritz pairs and estimates, 12 Ritz
 * vectors and residuals, 13 work queue.  Writes min(count, 14) entries and
 * returns that number. */
int rks_dbatch_phase_cycles(const rks_dbatch* b, int64_t* cycles, int count);

/* Ritz pairs of problem i, best first: returns nw (k, or k + 1 when a
 * complex pair straddles the cut) or a negative status; fills the first nw
 * entries of each non-NULL host array: eigenvalues, FP64 residuals, Rayleigh
 * quotients x^H A x / x^H x, estimates; X (n x nw host, LAPACK real packing
 * as rks_get_eigpairs) the Ritz vectors U y with ||y|| = 1. */
int rks_dbatch_eigpairs(rks_dbatch* b, int i, double* lam_re, double* lam_im, double* resid, double* rq_re,
                        double* rq_im, double* est, double* X);

/* Free the batch.  Safe on NULL. */
void rks_destroy_batched_dev(rks_dbatch* b);

/* ---- Sketch primitives (Sec. 5 setup; Def. 1.1) ---------------------- */

/* The (row, sign) pairs of Omega: for column i and slot t < zeta,
 * rows[i*zeta + t] in [0, d) and signs[i*zeta + t] in {-1, +1}.  Device
 * pointers (int32 and int8), written on `stream` (NULL: default stream).
 * Hash: base_i = mix(seed * 0x9E3779B97F4A7C15 + i); draw r =
 * mix(base_i + (r+1) * 0x9E3779B97F4A7C15), mix = SplitMix64's output
 * function; row = ((draw >> 32) * d) >> 32, sign = -1 if draw & 1; a draw
 * repeating an earlier row of the column is skipped; at most 32*zeta draws.
 * Requires d >= 2*zeta, 1 <= zeta <= 16. */
int rks_sketch_pairs(int64_t n, int d, int zeta, uint64_t seed, int32_t* rows, int8_t* signs,
                     void* stream);

/* z = Omega x for a device vector x (n doubles) into device z (d doubles),
 * entries sign/sqrt(zeta), FP64 accumulation.  Same requirements. */
int rks_sketch_apply(int64_t n, int d, int zeta, uint64_t seed, const double* x, double* z,
                     void* stream);

/* Largest sketch size d accepted by rks_sketch_apply_noalloc. */
#define RKS_NOALLOC_MAX_D 8192

/* z = Omega x exactly as rks_sketch_apply, but without allocating anything:
 * no cudaMalloc, cudaFree or allocating library call.  This has no
 * counterpart in the paper; it is for callers that cannot allocate device
 * memory, such as code running inside another framework's memory pool (which
 * already owns the device memory, so a private cudaMalloc can fail or
 * fragment it) or latency-critical loops that cannot pay the device-wide
 * synchronisation cudaFree implies.  Its scratch (d FP64 sums and a status
 * word) lives in one fixed device array of RKS_NOALLOC_MAX_D + 1 doubles that
 * every GPU loading the library holds until the process exits; d larger than
 * RKS_NOALLOC_MAX_D returns RKS_EINVAL.  The first call on a device (with that
 * device current) looks up the array's device address and caches it for the
 * process; the cached address is not valid after cudaDeviceReset.  All calls
 * share the array: the sums are cleared at the start of each call, and calls
 * that overlap on the GPU (different streams or host threads) race on it.
 * x: n doubles, z: d doubles, device pointers of the current device; z must
 * hold at least d doubles.  Every call copies a status word to the host and
 * synchronises `stream`, so it must not be called while `stream` is being
 * captured into a CUDA graph.  Returns RKS_OK, RKS_EINVAL (arguments, or the
 * hash draw cap reached) or RKS_ECUDA. */
int rks_sketch_apply_noalloc(int64_t n, int d, int zeta, uint64_t seed, const double* x, double* z,
                             void* stream);

/* ---- Restart product on the tensor cores (Eq. 3.5) ------------------ */

/* out = U Q for an FP32 basis, the restart product U_k = U Q' of the
 * mixed-precision path, on the tcgen05 tensor cores: U and Q are split into
 * three bf16 terms each, the six leading split products are accumulated in
 * FP32 (FP32-class accuracy).  out[i + o*ldu] = sum_l U[i + l*ldu] *
 * Q[l + o*nin] for i < n, o < nout.  U, out: device FP32 arrays with leading
 * dimension ldu >= n; out may equal U (each 128-row tile is read before it is
 * written).  Q: host FP64, nin x nout column-major, 1 <= nin <= 256,
 * 1 <= nout <= 64.  Runs on `stream` (NULL: default stream) and synchronises
 * it.  Returns RKS_OK, RKS_EINVAL (sizes, NULL pointers), RKS_ENOMEM,
 * RKS_ECUDA, or RKS_ETIMEOUT if a bounded device wait gave up. */
int rks_basis_product_f32(int64_t n, const float* U, int64_t ldu, int nin, const double* Q, int nout, float* out,
                          void* stream);

/* out = U Q as the double-float restart forms it on the tensor cores: every
 * row of U is a 47-bit fixed-point integer at the row's own power-of-two
 * scale, every column of Q one at the column's scale; both are cut into seven
 * digits (a signed top digit and six of 7 bits), whose 34 leading digit-pair
 * products are accumulated in FP32 (exactly where it matters) and recombined
 * in double-float, then FP64.  Accuracy: about 2^-46 of the row's largest
 * |U[i, l]| times sum_l |Q[l, o]|.  U, out: device FP64 arrays with leading
 * dimension ldu >= n (U is read as ldu x nin values and rounded to
 * double-float pairs); Q: host FP64, nin x nout column-major,
 * 1 <= nin <= 192, 1 <= nout <= 64, and the digit
 * image of Q must fit in shared memory (else RKS_EINVAL).  Allocates its
 * scratch, runs on `stream` and synchronises it.  Returns RKS_OK,
 * RKS_EINVAL, RKS_ENOMEM, RKS_ECUDA or RKS_ETIMEOUT. */
int rks_basis_product_df(int64_t n, const double* U, int64_t ldu, int nin, const double* Q, int nout, double* out,
                         void* stream);

/* ---- Randomized QR of a block (Sec. 2) -------------------------------- */

/* The randomized orthogonalisation processes Sec. 2 lists for building a
 * sketch-orthonormal basis, applied to a tall and skinny block K (n x s):
 * K = Q R with R upper triangular and a positive diagonal.
 *   RKS_QR_RGS      randomized Gram-Schmidt, column by column (the process of
 *                   Algorithm 2 without A): Omega Q orthonormal.
 *   RKS_QR_WHITEN   sketch and whiten (Sec. 3.3 on the whole block):
 *                   Omega K = Q_s R, Q = K R^{-1}: Omega Q orthonormal.
 *   RKS_QR_RCHOLQR  randomized Cholesky QR: whiten, then Cholesky QR of the
 *                   whitened block: Q orthonormal in the Euclidean sense.
 *   RKS_QR_RHQR     randomized Householder QR: Householder QR carried out in
 *                   the sketched space of Theta = [[I_s, 0], [0, Omega']],
 *                   where rows 0..s-1 are kept exactly and Omega' is the
 *                   sparse-sign embedding of dimension n - s for (d, zeta,
 *                   seed) on rows s..n-1; each reflector
 *                   H_j = I - beta_j u_j (Theta u_j)^T Theta is applied to the
 *                   columns, Q = H_0 ... H_{s-1} [I_s; 0]: Theta Q
 *                   orthonormal, stable for ill-conditioned K.
 * RGS and WHITEN compute the same (unique) factorisation in exact
 * arithmetic, RHQR the same with Theta in place of Omega, RCHOLQR the
 * Euclidean QR of K.  Omega is the solver's
 * sparse-sign embedding for (n, d, zeta, seed).  The n-dimensional work runs
 * in double-float arithmetic on the device, the d x s and s x s work in FP64
 * on the host. */
enum { RKS_QR_RGS = 0, RKS_QR_WHITEN = 1, RKS_QR_RCHOLQR = 2, RKS_QR_RHQR = 3 };
#define RKS_SKETCH_QR_MAX_S 192

/* K, Q: device FP64, column-major n x s with leading dimensions ldk, ldq >= n
 * (Q may be K, with ldq = ldk).  R: host s x s (column-major, ld s), written
 * with zeros below the diagonal.  S: host d x s or NULL; receives Omega Q
 * (measured by sketching the computed Q; for RGS the sketches the process
 * computed; for RHQR Omega' Q[s:, :], the sketched rows of Theta Q, whose
 * other rows are Q's first s rows).  RHQR needs n - s >= 2.  1 <= s <= min(RKS_SKETCH_QR_MAX_S, d, n), 1 <= zeta <= 16,
 * 2 zeta <= d <= 8192.  Work buffers (about 16 n s bytes) are allocated and
 * freed by the call; it runs on `stream` and synchronises it.  Returns
 * RKS_OK, RKS_EINVAL, RKS_ENOMEM, RKS_ECUDA, RKS_EBREAKDOWN (a zero or
 * non-finite diagonal of R: K is rank deficient) or RKS_EDENSE (RCHOLQR: the
 * Gram matrix is not positive definite). */
int rks_sketch_qr(int64_t n, int s, const double* K, int64_t ldk, int d, int zeta, uint64_t seed, int method,
                  double* Q, int64_t ldq, double* R, double* S, void* stream);

/* ---- Learned start vector for a parametric operator family ----------- */

/* The start vector u_1 of Algorithm 1 is drawn at random in the paper
 * (Sec. 2.1: it only needs components along the wanted eigenvectors).  For a
 * family of operators whose coefficient fields are known on an H x W grid
 * (the 2D convection-diffusion family: log nu, bx / 50, by / 50 as three
 * channels, channel-major, x fastest), a small network maps the fields to a
 * start vector close to the wanted invariant subspace.  It is a 4-level
 * U-Net: 15 3x3 convolutions (zero padding) of 32 channels (3 in, 1 out),
 * ReLU, 2x2 average pooling, 2x nearest upsampling, additive skip
 * connections; FP16 weights with FP32 masters, FP32 activations and
 * accumulation.  It is trained with the subspace-capture loss
 * L = 1 - ||Q^T u||^2 / ||u||^2, Q (n x q, n = H W) an orthonormal basis of
 * the wanted Schur vectors a solve of that operator returned (rks_get_schur),
 * by Adam.  A caller keeps a random component in the start vector and the
 * random start as the fallback; the residual of the solve judges it.
 * Parameters are one flat FP32 vector: for l = 1..15, W_l (cout x cin x 3 x 3,
 * row-major) then b_l (cout).  All device pointers are of the current device;
 * the calls run on the stream given at creation and synchronise it. */
typedef struct rks_ws rks_ws;

/* Number of parameters (121 409). */
int64_t rks_ws_nparams(void);

/* A network for H x W grids (H, W multiples of 8, H W <= 2^26) with He-normal
 * weights from SplitMix64(seed) and zero biases.  stream: cudaStream_t or
 * NULL (the network creates one).  Returns RKS_OK, RKS_EINVAL, RKS_ENOMEM or
 * RKS_ECUDA; on error *out is NULL. */
int rks_ws_create(rks_ws** out, int H, int W, uint64_t seed, void* stream);

/* Copy the FP32 master parameters to / from a host array of rks_ws_nparams
 * floats; set also clears the optimiser state and the accumulated gradient. */
int rks_ws_get_params(const rks_ws* s, float* theta);
int rks_ws_set_params(rks_ws* s, const float* theta);

/* u (device, H W floats) = the network applied to x (device, 3 x H x W). */
int rks_ws_forward(rks_ws* s, const float* x, float* u);

/* Forward, loss and backward for one sample: x (device, 3 x H x W), Q
 * (device FP32, n x q column-major, orthonormal columns, 1 <= q <= 64).  The
 * gradient of L is added to the network's accumulator; *loss (may be NULL)
 * receives L.  Returns RKS_ENAN if u = 0. */
int rks_ws_accumulate(rks_ws* s, const float* x, const float* Q, int q, double* loss);

/* The accumulated gradient (host, rks_ws_nparams floats); clear it. */
int rks_ws_get_grad(const rks_ws* s, float* grad);
int rks_ws_zero_grad(rks_ws* s);

/* One Adam step (beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected)
 * with the mean of the gradients accumulated since the last step, which are
 * then cleared.  RKS_ESTATE if nothing was accumulated. */
int rks_ws_adam_step(rks_ws* s, float lr);

/* The start vector for rks_create's opts.u1: u1 (device, H W doubles) =
 * u / ||u|| + eps g / ||g||, u the network's output for x (device,
 * 3 x H x W) and g the solver's own random start (N(0,1) entries from
 * SplitMix64(seed) and Box-Muller, as rks_create draws it from seed + 1):
 * the random component (eps, e.g. 1e-3) keeps every wanted direction present
 * whatever the network returns.  Norms in FP64.  RKS_ENAN if u = 0. */
int rks_ws_start_vector(rks_ws* s, const float* x, double eps, uint64_t seed, double* u1);

/* Free the network.  Safe on NULL. */
void rks_ws_destroy(rks_ws* s);

/* ---- Host-side small dense FP64 steps (Algorithm 1 contraction) ------ */

/* Ordered real Schur form (Prop. 2.8) of the m x m matrix B (column-major,
 * host): B = Q T Q^T with T quasi-triangular (standardised 2x2 blocks) and
 * the nsort best diagonal blocks for `which` leading, best first.  T and Q
 * are m x m host arrays.  Returns RKS_OK, RKS_EINVAL or RKS_EDENSE.  Runs on
 * the host only (no GPU needed). */
int rks_host_ordered_schur(int m, const double* B, int which, int nsort, double* T, double* Q);

/* Reorder a quasi-triangular T (n x n, column-major, host, in place) by
 * orthogonal swaps of adjacent diagonal blocks so that the blocks flagged in
 * select (n ints, read at each block's first row) lead, keeping the order of
 * the flagged blocks and of the others (the aggressive-deflation reorder,
 * Sec. 4.3).  Z (n x n, host) is multiplied on the right by the rotations
 * (pass the identity to get them).  Returns RKS_OK, RKS_EINVAL, or
 * RKS_EDENSE with T and Z unchanged when a swap is refused.  Host only. */
int rks_host_reorder_select(int n, double* T, const int* select, double* Z);

/* Eigenvalues and unit 2-norm eigenvectors of a quasi-triangular T (n x n,
 * host): a 2x2 block gives the pair (Im > 0 first).  Y_re, Y_im: n x n host
 * arrays (column j = eigenvector j).  Host only. */
int rks_host_quasi_eig(int n, const double* T, double* lam_re, double* lam_im, double* Y_re, double* Y_im);

/* Re-orthonormalisation of a drifted Krylov-Schur decomposition in the
 * sketch (the mixed path's hand-over to double-float; the whitening of
 * Sec. 3.3 with the last vector): A U = U T + u b^T with U of ka columns,
 * S = [Omega U, Omega u] (d x (ka+1), column-major, host, overwritten by Q of
 * S = Q R).  Returns Rinv = R^-1 ((ka+1) x (ka+1)) and the decomposition of
 * [V v] = [U u] R^-1: A V = V Tn + v bn^T, Tn = (R11 T + r12 b^T) R11^-1
 * (ka x ka), bn^T = r22 b^T R11^-1 (ka).  T: ka x ka, b: ka; all host.
 * Returns RKS_OK, RKS_EINVAL, or RKS_EDENSE if R is singular.  Host only. */
int rks_host_sketch_reorthonormalize(int d, int ka, double* S, const double* T, const double* b, double* Rinv,
                                     double* Tn, double* bn);

/* The device dense step of the persistent batched solver on one matrix
 * (test entry point): B (m x m, host, m <= 64) -> real Schur form T = Q^T B Q
 * whose leading blocks are the best blocks for `which` covering nsort
 * columns (pairs whole; in the order the Schur form had them): Algorithm 1's
 * Schur, reordering and truncation choice; then eigenvalues and unit
 * eigenvectors of T as rks_host_quasi_eig.  One warp on the current device,
 * double-float arithmetic (as in the solver); T, Q, Y_re, Y_im (m x m) and
 * lam_re, lam_im (m) host arrays (the last four may be NULL).  Returns RKS_OK,
 * RKS_EINVAL, RKS_EDENSE (no convergence of the QR iteration, or a refused
 * swap) or RKS_ECUDA. */
int rks_dev_ordered_schur(int m, const double* B, int which, int nsort, double* T, double* Q, double* lam_re,
                          double* lam_im, double* Y_re, double* Y_im);

#ifdef __cplusplus
}
#endif

#endif /* RKS_H */
