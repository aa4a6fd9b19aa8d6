/*
 * rcp.h -- C ABI of the GB300 (sm_103a) library for randomized complete pivoting (RCP):
 * the block LDL^T factorization  Pi^T A Pi = L D L^T  of a dense symmetric indefinite A
 * whose pivots come from a Gaussian sketch B = Omega A (Feng, Xiao and Gu,
 * "Randomized complete pivoting for solving symmetric indefinite linear systems").
 *
 * Layout and conventions (all entry points):
 *   - Matrices are column-major with a leading dimension (lda >= n).  Only the LOWER
 *     triangle of a symmetric matrix is read or written.
 *   - perm[i] (0-based) is the original index of the row/column that ends at position i:
 *     A(perm[i], perm[j]) = (L D L^T)(i, j).
 *   - L is unit lower triangular and is returned in the strictly lower triangle of the
 *     factored array (its unit diagonal is implicit).  D is block diagonal with 1x1 and
 *     2x2 blocks: Dd[i] = D(i, i), Ds[i] = D(i+1, i) (0 for a 1x1 block and for i = n-1).
 *   - Device pointers are marked "device"; the caller owns every buffer it passes in.
 *     A handle owns only its workspace (sketch, panels, status words), allocated with
 *     cudaMalloc on first use and grown when a larger problem arrives; it is freed by
 *     rcp_destroy.  One handle serves one stream at a time.
 *   - Every call is asynchronous on the given stream unless it fills a host rcp_stats,
 *     in which case it synchronizes that stream before returning.  The host-driven calls
 *     synchronize always (and cannot be captured in a graph): rcp_refine_gmres, rcp_factor
 *     and rcp_sysv with the Algorithm 2 safeguard (opts->guard_r > 0, once per panel),
 *     rcp_l_norms, rcp_exchange_latency and rcp_wait_expiry.
 *
 * Errors: a negative rcp_status is returned before anything is launched when an argument
 * is invalid.  Numerical faults found on the device (non-finite values, a bounded wait
 * that ran out) are recorded in the handle's device status word and reported by the next
 * call that synchronizes (any call given a non-NULL stats, or rcp_sync).  A positive
 * value is LAPACK's info: 1 + position of the first 1x1 pivot that is exactly zero; the
 * factorization still completes.  No kernel of this library traps or asserts.
 */
#ifndef RCP_GB300_H
#define RCP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rcp_stream_t;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    RCP_OK = 0,
    RCP_EINVAL = -1,        /* invalid argument                                    */
    RCP_ENOMEM = -2,        /* workspace allocation failed                         */
    RCP_ECUDA = -3,         /* a CUDA runtime call failed                          */
    RCP_ENONFINITE = -4,    /* NaN or Inf met in a pivot or a norm                 */
    RCP_ETIMEOUT = -5,      /* a bounded device-side wait ran out                  */
    RCP_ENOCONV = -6,       /* refinement did not reach the tolerance in max_iter  */
    RCP_EUNSUPPORTED = -7   /* size or option combination not supported            */
} rcp_status;

typedef enum {
    RCP_FP64 = 0,           /* everything in FP64 (CUDA cores)                             */
    RCP_FP32 = 1,           /* FP32 factor; FP32 trailing update on CUDA cores                  */
    RCP_TF32 = 2,           /* reserved: currently runs as RCP_FP32                              */
    RCP_TF32X3 = 3,         /* FP32 factor; sketch B = Omega A and trailing update on tcgen05   */
                            /* tensor cores with split TF32 operands (hi*hi + hi*lo + lo*hi,    */
                            /* FP32 accumulation)                                               */
    RCP_F16X3 = 4           /* as RCP_TF32X3, the trailing update's split in FP16 (the same 11  */
                            /* significant bits per part; the sketch keeps split TF32, which    */
                            /* needs no scaling): W and L21 are scaled by powers of two so that */
                            /* their panel maxima sit below 2^15, the three products run at the */
                            /* FP16 tensor rate and move half the operand bytes of TF32         */
} rcp_prec;

typedef struct {
    int b;              /* panel width (block size of Algorithm 1); 0 = default 64           */
    int d;              /* sketch rows (the paper's p; 1..128); 0 = default min(b + 16, 128) */
    int q_mode;         /* 1 (or 0): q = 1, one sketch argmax and one sketch update per      */
                        /* pivot step.  2: q = b (Section 3.1): a b-step partial QRCP of the */
                        /* sketch picks each block's candidates, the block's steps take them */
                        /* in order (SBKP may still bring in other columns), and the sketch  */
                        /* is updated once per block, B(:, k1:n) -= B_blk L11^{-T} L21^T.    */
                        /* rcp_factor_batched supports q = 1 only, without the safeguard.     */
    uint64_t seed;      /* Philox key of the sketch matrix Omega                             */
    rcp_prec prec;      /* arithmetic of the factor                                          */
    double alpha;       /* SBKP threshold; 0 = default sqrt(2)/2                             */
    const void *omega;  /* optional device d x n Omega (ld = d) in the factor precision;     */
                        /* NULL = draw it from Philox(seed)                                  */
    int grid;           /* CTAs of the persistent panel kernel; 0 = automatic                */
    int guard_r;        /* Algorithm 2 safeguard, q = 1 only (0 = off, Algorithm 1 as is):   */
                        /* with beta = ||B^(1)||_{1,2} and delta = (j+1)/r after j sketch    */
                        /* recomputations, a pivot whose sketch column norm t falls below   */
                        /* eps^delta beta ends the panel; while j + 1 < r a fresh Omega'    */
                        /* (Philox stream j + 1 of seed, d x (n-k)) re-sketches the Schur     */
                        /* complement and the check is repeated with the larger delta; else  */
                        /* the factorization stops: the Schur complement counts as zero      */
                        /* (D(k:n) = 0, L(k:n, k:n) = I, info = k + 1, stats->rank = k).     */
                        /* The host reads the state after every panel: the call synchronizes */
                        /* once per panel and cannot be captured in a graph.  1 <= r <= 64.  */
    double guard_eps;   /* eps of the safeguard; 0 = machine epsilon of the factor (2^-52    */
                        /* FP64, 2^-23 otherwise)                                             */
} rcp_opts;

typedef struct {
    double growth_D;          /* rho = max|D_ij| / max|A_ij|  (experiments section)         */
    double max_abs_L;         /* max |L_ij|, i > j                                          */
    double min_sketch_ratio;  /* min over steps of ||B(:, pi_k)|| / ||B^(1)||_{1,2}          */
    int n_2x2;                /* number of 2x2 pivot blocks                                 */
    int info;                 /* LAPACK-style zero-pivot position (1-based), 0 if none      */
    int refine_iters;         /* refinement corrections applied (rcp_refine)                */
    int device_flags;         /* raw device status bits                                     */
    double berr;              /* final normwise backward error (rcp_refine)                 */
    double anorm;             /* ||A||_inf of the original matrix (rcp_refine)              */
    int gmres_iters;          /* GMRES iterations (applications of M^{-1} A) of              */
                              /* rcp_refine_gmres, or of rcp_sysv's fallback to it          */
    int rank;                 /* rcp_factor with the safeguard: columns eliminated before a  */
                              /* rank-deficiency stop (n when it did not stop)               */
    int resketches;           /* rcp_factor with the safeguard: sketch recomputations        */
} rcp_stats;

typedef struct rcp_handle rcp_handle;

/* Create / destroy a handle.  rcp_create allocates no device memory. */
rcp_status rcp_create(rcp_handle **h);
void rcp_destroy(rcp_handle *h);

/* Human-readable name of a status code (static string). */
const char *rcp_status_string(int status);

/* Wait for the handle's stream work and report the device status word (0 = fine). */
rcp_status rcp_sync(rcp_handle *h, rcp_stream_t stream);

/* Size the workspace for order n and the given options without factoring, so that a
 * later call makes no allocation (needed before capturing calls in a CUDA graph). */
rcp_status rcp_reserve(rcp_handle *h, int n, int nrhs, const rcp_opts *opts);

/*
 * rcp_factor -- Algorithm 1 (blocked RCP, q = 1): draw Omega (d x n, Philox4x64-10 and
 * Box-Muller), form B = Omega A, then per block of b columns: per pivot step the
 * column-norm argmax on B, the symmetric interchange, the SBKP 1x1/2x2 choice
 * (Figure SBKP, alpha = sqrt(2)/2), the multipliers L21 = A21 A11^{-1} (2x2 inverses in
 * FP64), the sketch update B(:, k+s:n) -= B(:, k:k+s-1) L(k+s:n, k:k+s-1)^T
 * (Eq. "Update matrix B"); after the block the deferred trailing update A22 -= W L21^T.
 *
 *   n            order (n >= 0; n = 0 is a no-op)
 *   A, lda       device, n x n lower triangle; double* when opts->prec == RCP_FP64, float*
 *                otherwise.  In: A.  Out: L in the strictly lower triangle (rows and columns
 *                permuted), the diagonal overwritten by D's diagonal.
 *   Dd, Ds       device double[n]: D's diagonal and sub-diagonal
 *   perm         device int[n]: the permutation (see conventions)
 *   opts         options (NULL = defaults: FP64, b = 64, d = 80, seed 0)
 *   stream       CUDA stream
 *   stats        host, filled after a stream synchronization; NULL = stay asynchronous
 * Returns RCP_OK, a negative error, or info > 0 (only when stats != NULL).
 */
rcp_status rcp_factor(rcp_handle *h, int n, void *A, int lda, double *Dd, double *Ds, int *perm,
                      const rcp_opts *opts, rcp_stream_t stream, rcp_stats *stats);

/*
 * rcp_solve -- solution phase (operation-count table, "solution phase"):
 * X <- Pi L^{-T} D^+ L^{-1} Pi^T X for nrhs right-hand sides, D^+ the pseudo-inverse of D (a
 * zero 1x1 block contributes 0: the basic solution when D is singular).
 *   LA, lda      device factor from rcp_factor (double* for RCP_FP64, float* otherwise)
 *   Dd, Ds, perm device, from rcp_factor
 *   prec         the precision the factor was computed in
 *   X, ldx       device double, n x nrhs: right-hand sides in, solutions out.  For an FP32
 *                factor the solve runs in FP32 and X is rounded through FP32.
 */
rcp_status rcp_solve(rcp_handle *h, int n, int nrhs, const void *LA, int lda, const double *Dd,
                     const double *Ds, const int *perm, rcp_prec prec, double *X, int ldx,
                     rcp_stream_t stream);

/*
 * rcp_refine -- FP64 iterative refinement on top of a (possibly FP32) factor:
 * x_0 = solve(b); repeat r = b - A x (FP64, original A), berr = ||r||_inf /
 * (||A||_inf ||x||_inf) (the experiments section's backward error), stop when berr <= tol,
 * else x += solve(r).  At most max_iter corrections; the loop also stops when a correction
 * fails to halve berr (the factor's error times the condition number is not small: the
 * iteration stagnates or diverges; rcp_refine_gmres is the remedy).  Without stats the loop
 * control stays on the device (no host round trip per iteration: all max_iter iterations are
 * launched and those after the stop skip their work, so the call can be captured); with stats
 * (the call synchronizes anyway) the host reads the stop flag after each check and launches no
 * further iterations.
 *   A64, lda     device double: the ORIGINAL matrix (lower triangle)
 *   LA, ldla     device factor; Dd, Ds, perm from rcp_factor; prec its precision
 *   Bv, ldb      device double n x nrhs right-hand sides
 *   X, ldx       device double n x nrhs, output solutions
 *   stats        host; when non-NULL: berr (max over columns), refine_iters, anorm; returns
 *                RCP_ENOCONV if berr > tol after max_iter corrections
 */
rcp_status rcp_refine(rcp_handle *h, int n, int nrhs, const double *A64, int lda, const void *LA,
                      int ldla, const double *Dd, const double *Ds, const int *perm, rcp_prec prec,
                      const double *Bv, int ldb, double *X, int ldx, double tol, int max_iter,
                      rcp_stream_t stream, rcp_stats *stats);

/*
 * rcp_refine_gmres -- GMRES-based iterative refinement (Carson and Higham, "Accelerating the
 * solution of linear systems by iterative refinement in three precisions", 2018): per outer
 * step r = b - A x (FP64, original A), stop when berr <= tol (as rcp_refine), else solve the
 * correction equation A d = r by one cycle of at most `restart` steps of GMRES (Saad and
 * Schultz, 1986) on the left-preconditioned system M^{-1} A d = M^{-1} r, M = L D L^T the
 * computed factor (applied by rcp_solve's kernels), FP64 Krylov basis with classical
 * Gram-Schmidt applied twice, until the preconditioned residual falls by 1e-10; x += d.
 * Converges where the factor is too inaccurate for rcp_refine: with FP32 factors it reaches
 * berr <= 1e-12 on matrices with condition numbers up to about 1e10 (beyond that, factor in
 * FP64).  Right-hand sides are refined one after another.
 *   arguments as rcp_refine; restart: Krylov dimension per cycle (0 = 64, at most 128);
 *   max_outer: corrections (GMRES cycles) per right-hand side; use_x != 0: X holds the starting
 *   iterates, else X = solve(B) first.
 *   stats (host, optional): berr (max over columns), refine_iters (cycles), gmres_iters
 * The host takes the scalars of each GMRES step (one device-to-host read per step), so the
 * call synchronizes the stream and cannot be captured in a graph.  Returns RCP_ENOCONV when
 * berr > tol after max_outer cycles.
 */
rcp_status rcp_refine_gmres(rcp_handle *h, int n, int nrhs, const double *A64, int lda, const void *LA,
                            int ldla, const double *Dd, const double *Ds, const int *perm, rcp_prec prec,
                            const double *Bv, int ldb, double *X, int ldx, double tol, int max_outer,
                            int restart, int use_x, rcp_stream_t stream, rcp_stats *stats);

/* Host helper of rcp_refine_gmres (no device work): y = argmin || beta e_1 - H y ||_2 for the
 * (k+1) x k upper Hessenberg H (column-major, ldh >= k+1; entries below the subdiagonal are
 * ignored), by Givens rotations; *resid = the minimal residual norm.  A zero diagonal after
 * the rotations (singular H) gives y_j = 0. */
rcp_status rcp_gmres_lsq(int k, const double *H, int ldh, double beta, double *y, double *resid);

/*
 * rcp_sysv -- solve A X = B end to end: copy the lower triangle of A64 (rounding it to
 * FP32 for the mixed precisions) into handle workspace, rcp_factor, rcp_refine; when that
 * stops short of tol (stagnation), rcp_refine_gmres from its iterate (stats->gmres_iters > 0).
 *   A64, lda, Bv, ldb, X, ldx   device pointers, or host pointers when host_buffers != 0 (then
 *                the copies in and out are part of the call; pinned host memory is fastest; of
 *                A64 only the lower triangle is transferred, as rectangles of 256 columns from
 *                each block's diagonal down: sum over blocks of (n - j0) x 256 doubles)
 *   tol, max_iter               refinement control (max_iter = 0: plain solve, no refinement)
 *   stats                       host, required (the call synchronizes)
 */
rcp_status rcp_sysv(rcp_handle *h, int n, int nrhs, const double *A64, int lda, const double *Bv,
                    int ldb, double *X, int ldx, const rcp_opts *opts, double tol, int max_iter,
                    int host_buffers, rcp_stream_t stream, rcp_stats *stats);

/*
 * Phase timing (off by default).  With profiling on, every call brackets each phase's
 * launches with two CUDA events on its stream; rcp_profile_read waits for them and returns,
 * per phase, the summed milliseconds and the number of bracketed stretches since the last
 * read.  Phases: 0 sketch (Omega + B = Omega A), 1 panel, 2 interchange, 3 trailing update,
 * 4 solve (forward, D, backward), 5 residual (refinement), 6 the host-to-device copies of
 * rcp_sysv with host buffers (on the stream that issues them; for FP32 factors a second stream,
 * where they overlap phase 0).  Profiling adds event records between launches, so time calls
 * with it off.
 */
rcp_status rcp_profile(rcp_handle *h, int enable);

/* How the FP32 panel speculates on SBKP case (1) of the next pivot step while it waits at a pivot
 * step's grid barrier (an implementation choice; Algorithm 1 has no counterpart, and every mode
 * gives bit-identical factors): -1 automatic (the default: with a shadow copy of the CTA's sketch
 * columns when it fits in shared memory, else with the confirmed sketch update deferred to the next
 * step's pass), 0 off (two grid exchanges per pivot step), 1 shadow copy, 2 deferred update.  A
 * forced mode whose shared memory does not fit makes the factorization return RCP_EUNSUPPORTED.
 * Applies to the handle's later FP32 factorizations with q = 1; RCP_EINVAL for other values. */
rcp_status rcp_set_speculation(rcp_handle *h, int mode);

/* With rcp_profile(h, 2), the next factorizations also record, for every pivot position k,
 * sixteen SM clock stamps (clock64 of one thread of the first CTA) at fixed points of the panel
 * step (top, before/after barrier 1, Schur column P, before/after barrier 2, decision, column r,
 * multipliers, sketch update, and inside the argmax and the committed speculation).
 * rcp_panel_trace copies up to cap stamps (16 per position, zero where a step started at
 * another position or a point was not reached) of the last such factorization. */
rcp_status rcp_panel_trace(rcp_handle *h, unsigned long long *out, int cap);

/* Latency floor of the FP32 panel's pivot step: `rounds` rounds of its grid-wide exchange
 * (each CTA adds a packed key to a ring slot by red.max, grid barrier, read-back) on `grid`
 * cooperative CTAs of the panel's 512 threads (0 = one per SM), without the step's arithmetic,
 * timed with CUDA events on `stream` after a short warm-up; *us = microseconds per round.
 * Uses the handle's barrier and key buffers (not while a factorization runs on the handle);
 * synchronizes the stream. */
rcp_status rcp_exchange_latency(rcp_handle *h, int grid, int rounds, rcp_stream_t stream, double *us);

/* Failure path of the bounded device waits: one cooperative launch of `grid` CTAs of the panel's
 * 512 threads (0 = one per SM) in which every CTA waits at a grid barrier for one arrival more
 * than the launch has CTAs, so that no wait can complete.  Each CTA gives up after limit_us
 * microseconds (1 .. 2000000; the library's own waits give up after 2 s), records a timeout in
 * the handle's status word and returns: no kernel hangs or traps.  *waited_us = how long the
 * first CTA waited.  Synchronizes the stream and returns what rcp_sync then reports, i.e.
 * RCP_ETIMEOUT; the status word stays set until a call that starts a factorization clears it,
 * and the handle remains usable. */
rcp_status rcp_wait_expiry(rcp_handle *h, int grid, int limit_us, rcp_stream_t stream, double *waited_us);

/* Stability diagnostics of a factor (the paper's experiments report them per matrix type):
 * *norm1_L = ||L||_1 exactly (unit lower L from rcp_factor: LA's strictly lower triangle, unit
 * diagonal), *norm1_Linv = an estimate of ||L^{-1}||_1 by Higham's 1-norm estimator (1988; a
 * lower bound, usually exact), from at most six solves with L and L^T.  prec: the precision of
 * LA.  Synchronizes the stream. */
rcp_status rcp_l_norms(rcp_handle *h, int n, const void *LA, int lda, rcp_prec prec, rcp_stream_t stream,
                       double *norm1_L, double *norm1_Linv);

/* Number of kernels this library has launched in the process so far (all handles). */
long long rcp_kernel_launches(void);
rcp_status rcp_profile_read(rcp_handle *h, double *ms, int *launches, int nphase);

/*
 * Batched ragged systems: many independent symmetric systems A_i x_i = b_i of small order
 * (n_i <= nmax, typically 32..512), each factored by Algorithm 1 (q = 1) exactly as rcp_factor
 * does, and solved or refined exactly as rcp_solve / rcp_refine do.  One persistent kernel per
 * phase covers the whole batch (the factor: two with a split schedule, see
 * rcp_set_batched_schedule): one CTA works on one system at a time, taking systems from an
 * atomic ticket in decreasing order of n_i; the sketch and the current panel of a system live
 * in that CTA's shared memory, A_i in global memory.  No call allocates memory once the handle's
 * batch workspace (order array, ticket, Omega, per-CTA scratch: about 4 * (batch + nmax) +
 * 8 * d * nmax bytes plus the scratch) is large enough, so after one warm-up call with the same
 * batch, nmax and schedule the calls can be captured into a CUDA graph.
 *
 * Pointer arrays ("device array of device pointers") hold one pointer per system; every other
 * per-system array is a device array of length batch.  nmax (host) bounds every n_i; systems
 * with n_i outside [0, nmax] are not processed correctly and must not be passed.
 *
 * rcp_factor_batched -- P_i^T A_i P_i = L_i D_i L_i^T for every system.
 *   A[i]    device, n_i x n_i, ld lda[i], lower triangle; overwritten by L_i (strictly lower,
 *           unit diagonal implicit) with D_i(j, j) on the diagonal.  Element type: double for
 *           RCP_FP64, float for every other opts->prec (the batched factor runs on CUDA cores;
 *           RCP_TF32X3, RCP_F16X3 and RCP_TF32 run as RCP_FP32 here).
 *   A64     optional (NULL allowed) device array of pointers to FP64 originals (ld lda64[i]):
 *           their lower triangles are first copied (rounded) into A[i] by the same kernel.
 *   Dd, Ds, perm: per-system outputs with the meaning they have for rcp_factor.
 *   opts    b (0: the shape chosen by rcp_tune_batched for this nmax/d/precision, else 32),
 *           d (0: b + 8, or the d tuned with b; at most 128), seed, alpha, omega as for
 *           rcp_factor; one Omega (d x nmax) serves every system, system i using its first
 *           n_i columns (the same columns a d x n_i draw with that seed gives).  q_mode 1 only.
 *   info    device [batch]: 0, or 1 + position of the first exactly-zero 1x1 pivot, or -4
 *           (RCP_ENONFINITE) when the system met a NaN or Inf (its factor is then incomplete).
 *   Returns RCP_EUNSUPPORTED when the shared-memory state of one system, (d + 2 (b + 1) + 2)
 *   * nmax + 2 d elements (4 or 8 bytes), does not fit one CTA (nmax = 512 at the defaults
 *   in FP32, 256 in FP64).  Asynchronous.
 *
 * rcp_refine_batched -- x_i = solve(b_i), then, when A64 != NULL, FP64 iterative refinement
 *   (r = b - A x in FP64, berr as rcp_refine, x += solve(r)) until berr_i <= tol or max_iter
 *   corrections.  Right-hand sides are processed 16 at a time; each group iterates on its own
 *   and iters[i] is the largest count of a group.
 *   LA/ldla: factors from rcp_factor_batched (prec RCP_FP64: double, else float).
 *   Bv/ldb:  right-hand sides (n_i x nrhs, FP64); X/ldx: solutions (n_i x nrhs, FP64); X must
 *            not overlap Bv.
 *   berr, iters: device [batch] or NULL; berr is 0 when A64 is NULL.
 *   The convergence test is per system; systems that miss the tolerance are not an error of
 *   the call: compare berr with tol.  Asynchronous.
 */
rcp_status rcp_factor_batched(rcp_handle *h, int batch, int nmax, const int *n, const double *const *A64,
                              const int *lda64, void *const *A, const int *lda, double *const *Dd,
                              double *const *Ds, int *const *perm, const rcp_opts *opts, int *info,
                              rcp_stream_t stream);
/* rcp_tune_batched -- autotuner of the batched factor: times rcp_factor_batched on the caller's
 *   batch (A64 required: every trial re-copies the originals into A) for every panel width b in
 *   {8, 12, 16, 24, 32, 48, 64} whose per-system state fits one CTA's shared memory, each with
 *   the CTA schedules of rcp_set_batched_schedule: (512, 0), (256, 0) where two 256-thread CTAs
 *   fit an SM, (128, 0) where three 128-thread CTAs do, and (512, min(256, nmax / 2)), and keeps
 *   the fastest shape and schedule for
 *   (nmax, opts->d, FP64 or not) in the handle: later rcp_factor_batched calls with opts->b == 0
 *   and the same opts->d use them.  With opts->d > 0 the width changes only the
 *   blocking of the deferred trailing update (with q = 1 the pivot sequence is the same in exact
 *   arithmetic).  With opts->d == 0 the sketch follows the width, d = b + 8 (Algorithm 1's
 *   d = b + p with oversampling p = 8), and the pair (b, d) is tuned together.  Synchronizes the
 *   stream; not for use during stream capture.  best_b / best_ms (host, may be NULL) get the
 *   chosen width and its factor time; rcp_get_batched_schedule reports the whole choice. */
rcp_status rcp_tune_batched(rcp_handle *h, int batch, int nmax, const int *n, const double *const *A64,
                            const int *lda64, void *const *A, const int *lda, double *const *Dd,
                            double *const *Ds, int *const *perm, const rcp_opts *opts, int *info,
                            rcp_stream_t stream, int *best_b, float *best_ms);
/* rcp_set_batched_schedule -- how later rcp_factor_batched calls on this handle spread the systems
 *   over CTAs (a deployment choice; the paper, whose experiments factor one system at a time, has
 *   no counterpart).  Each CTA factors one system at a time and the factor is bound by the latency
 *   of each pivot step, so two resident CTAs per SM overlap two systems' waits.
 *   threads 512: one launch of 512-thread CTAs (one per SM);  threads 256 or 128: one launch of
 *   256- or 128-thread CTAs, as many per SM as their shared state and registers allow (up to two
 *   or four);  split > 0 (threads 0 or 512): systems with n_i > split in a launch of 512-thread
 *   CTAs, then those with n_i <= split in a launch of 256-thread CTAs whose shared state is sized
 *   for order split.  The schedule changes
 *   which thread does what, not the arithmetic of a system, except that an FP32 system whose
 *   launch keeps its sketch in registers (d <= 48 and the launch's order <= its CTA size) rounds
 *   the 2x2 steps' sketch update in another order than one that keeps it in shared memory.
 *   threads = split = 0 (the default): the schedule chosen by rcp_tune_batched, else (512, 0).
 *   RCP_EINVAL for other values (threads not 0, 128, 256 or 512; split < 0; split > 0 with threads
 *   128 or 256).
 * rcp_get_batched_schedule -- the shape (b, d) and schedule (threads, split) that rcp_factor_batched
 *   would use for (nmax, d, prec) with opts->b == 0 (d = 0 as in rcp_opts).  Host outputs may be
 *   NULL. */
rcp_status rcp_set_batched_schedule(rcp_handle *h, int threads, int split);
rcp_status rcp_get_batched_schedule(rcp_handle *h, int nmax, int d, rcp_prec prec, int *b, int *d_out,
                                    int *threads, int *split);
rcp_status rcp_refine_batched(rcp_handle *h, int batch, int nmax, int nrhs, const int *n,
                              const double *const *A64, const int *lda64, const void *const *LA,
                              const int *ldla, const double *const *Dd, const double *const *Ds,
                              const int *const *perm, rcp_prec prec, const double *const *Bv, const int *ldb,
                              double *const *X, const int *ldx, double tol, int max_iter, double *berr,
                              int *iters, rcp_stream_t stream);

/*
 * Building blocks exposed for testing.
 * rcp_omega:  Omega (d x n, ld d, FP64, device) from Philox4x64-10: entries (2t, 2t+1) of
 *             column j come from counter (j, t, 0, 0) and key (seed, 0) through Box-Muller
 *             (u1 = (w0 >> 11 + 1) 2^-53, u2 = (w1 >> 11) 2^-53).  Section 3, "draw Omega".
 * rcp_sketch: B = Omega A (d x n, ld d, device, precision prec) for the lower-stored
 *             symmetric A; Omega drawn from seed unless omega != NULL.  Section 3, B = Omega A.
 *             RCP_FP64 and RCP_FP32 run on the CUDA cores; RCP_TF32X3 and RCP_F16X3 on the
 *             tcgen05 tensor cores with split TF32 operands (hi*hi + hi*lo + lo*hi, FP32
 *             accumulation), as rcp_factor forms the sketch in those precisions.
 */
rcp_status rcp_omega(int d, int n, uint64_t seed, double *omega, rcp_stream_t stream);
rcp_status rcp_sketch(int n, int d, const void *A, int lda, rcp_prec prec, uint64_t seed,
                      const void *omega, void *B, rcp_stream_t stream);

/*
 * rcp_solve_noalloc -- the same solve as rcp_solve for callers that cannot allocate device
 * memory when they solve: hard real-time loops that must never block in the allocator, and
 * programs whose device memory belongs to another allocator (a framework's pool, an embedding
 * application with a fixed memory budget).  It takes no handle and calls no cudaMalloc,
 * cudaFree or allocating library routine; its scratch is one 16 MiB array in device memory
 * that every GPU loading this library keeps until the process exits.
 * (The paper has no counterpart to this entry point; it is a deployment convenience.)
 *   Arguments, layout and results are those of rcp_solve.
 *   Limit, with nb = ceil(n / 64), sizes in bytes, each term rounded up to 256:
 *     FP64 factor:  8 n nrhs + 32768 nb + 4 (2 nb + 3)             <= 16 MiB
 *     FP32 factors: 16 n nrhs + 4 n nrhs + 49152 nb + 4 (2 nb + 3) <= 16 MiB
 *   e.g. n = 16384: nrhs <= 63 for an FP64 factor, nrhs <= 12 for an FP32 one.  Larger problems
 *   return RCP_EUNSUPPORTED before anything is launched.
 *   The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 *   not stream-ordered): make that first call before any stream capture.
 *   All calls share the array and it keeps the last call's contents: each call clears, on its
 *   stream, the parts that must start at zero.  Calls whose kernels can overlap on the GPU
 *   (different streams, or unsynchronized host threads) race and give wrong results.
 *   The call is asynchronous and returns only argument and launch errors.  A failure found on
 *   the device (a bounded wait that ran out, a non-finite diagonal block of L) fills X with NaN.
 */
rcp_status rcp_solve_noalloc(int n, int nrhs, const void *LA, int lda, const double *Dd, const double *Ds,
                             const int *perm, rcp_prec prec, double *X, int ldx, rcp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* RCP_GB300_H */
