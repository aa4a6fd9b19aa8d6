// kernels.h -- launchers of the RCP kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rcpk {

// clock64 stamps per pivot position in the panel trace (profiling level 2)
constexpr int PANEL_TRACE_SLOTS = 16;
// 64-bit words of the FP32 panel's argmax key rings (pivot keys, then speculative keys).  A ring
// slot is indexed by the grid-barrier generation and cleared half a ring ahead of its use, which
// assumes consecutive generations: a cooperative kernel that advances the generation without the
// panel's clearing (the block QRCP) zeroes all of them.
constexpr int PANEL_KEY_WORDS = 512;   // two key rings of 16 slots, one 128-byte line per slot

// Omega (d x n) from Philox counter (j, t, stream, 0) and key (seed, 0)
template <typename T>
cudaError_t launch_omega(int d, int n, uint64_t seed, T *om, cudaStream_t s, uint64_t stream = 0);

// B = Omega A (d x n).  In FP32, `part` (nullable, part_elems elements) holds the partial sums
// of a split over K; sketch_scratch_floats(n, d) elements allow the full split.
template <typename TA, typename TC>
cudaError_t launch_sketch(int n, int d, const TA *A, int lda, const TC *om, TC *B, TC *part, size_t part_elems,
                          cudaStream_t s);
size_t sketch_scratch_floats(int n, int d);
// B(:, c0:c1) = sum over S slices of part (slice order), count = d (c1 - c0)
cudaError_t launch_sketch_reduce(size_t count, int S, const float *part, float *B, cudaStream_t s);

// Tensor-core sketch (split TF32 on tcgen05) for the FP32 factors of RCP_TF32X3 / RCP_F16X3:
// Omega is first split into swizzled tiles (sketch_tc_omega_floats(n, d) floats), then columns
// c0 .. c1-1 of B = Omega A are formed (A must hold its final values in columns < c1); `part`
// holds sketch_tc_scratch_floats(n, d) floats of slice partial sums; a bounded wait that runs
// out sets ST_TIMEOUT in *status.
int sketch_tc_slices(int n);
size_t sketch_tc_omega_floats(int n, int d);
size_t sketch_tc_scratch_floats(int n, int d);
cudaError_t launch_omega_split(int n, int d, const float *om, float *omt, cudaStream_t s);
cudaError_t launch_sketch_tc(int n, int d, const float *A, int lda, const float *omt, float *B, float *part,
                             size_t part_floats, int c0, int c1, int *status, cudaStream_t s);

// Per-factorization workspace pointers used by the panel / interchange / trailing kernels.
template <typename T>
struct FactorWork {
    int n, lda;
    T *A;               // the matrix being factored (lower storage)
    int d;
    T *B;               // sketch, d x n, ld d
    int bmax, bw;       // panel width target and row stride of the panel buffers (bmax + 1)
    double alpha;
    T *Wbuf;            // n x bw, column-major (ld n): W = L D rows of the panel, logical order
    T *Lc;              // n x bw, column-major (ld n), position order: the panel's multipliers
    T *Lg;              // n x bw, row-major by block-start index: multipliers as they are made
    double *Dd, *Ds;
    int *perm;
    int *lpos;          // [n]: final position in the panel of each block-start index
    int *moved;         // [n]: block-start indices whose position changed
    FactorState *st;
    double *s1v, *s2v;  // reduction slots
    int *s1i, *s2i;
    T *pay;             // [2][grid][d] sketch column of each CTA's candidate
    unsigned *bar;
    int *status;
    int grid;           // CTAs of the cooperative panel kernel
    int chunk_cap;      // max columns per CTA
    // interchange scratch
    T *tmpA;            // [maxmoved][n]
    T *tmpL;            // [maxmoved][n]
    int *tmpP;          // [maxmoved]
    int maxmoved;
    unsigned long long *trace;   // optional per-step timestamps (profiling), 10 per position
    unsigned long long *keys;    // ring of packed argmax keys (FP32 path), zeroed per factorization
    float *tcops;                // tensor-core operand tiles (TF32x3 trailing update)
    int spec;                    // FP32 panel: speculative case-(1) path enabled (shadow sketch fits)
    double *s3v;                 // [2][grid][4] records of the speculative candidates
    int *psnap;                  // [panels][n]: perm after each panel (deferred L-row interchanges)
    int *pinv;                   // [panels][n]: their inverses
    int *pbounds;                // [panels][2]: (k0, kend) of each panel
    int qb;                      // Algorithm 1 with q = b: the pivot of step k is the column at
                                 // position k (candidates chosen by the block QRCP); no per-step
                                 // sketch update (the block update follows the panel)
    int guard_r;                 // Algorithm 2 safeguard: r (0 = off)
    double guard_eps;            //   and its eps
};

template <typename T>
size_t panel_smem_bytes(int d, int bw, int chunk_cap, int spec);

// q = b: block QRCP of the sketch (interchanges in the panel's format) and block sketch update
template <typename T>
size_t qrcp_smem_bytes(int d, int chunk_cap);
size_t qrcp_smem_limit();
template <typename T>
cudaError_t launch_qrcp(const FactorWork<T> &w, int steps, cudaStream_t s);
template <typename T>
cudaError_t launch_block_sketch_update(const FactorWork<T> &w, T *ytmp, cudaStream_t s);
// Y = B(:, k0:k1) L11^{-T} (d x nb, ld d) of the panel just done, into ytmp
template <typename T>
cudaError_t launch_bsk_y(const FactorWork<T> &w, T *ytmp, cudaStream_t s);
// the block sketch update on tcgen05 (split TF32): Y, its tiles (block_update_tc_floats(bw, d)
// floats in ytiles), then B(:, k1:n) -= Y L21^T
size_t block_update_tc_floats(int bw, int d);
cudaError_t launch_block_sketch_update_tc(const FactorWork<float> &w, float *ytmp, float *ytiles, cudaStream_t s);

template <typename T>
cudaError_t launch_panel(const FactorWork<T> &w, cudaStream_t s);

template <typename T>
cudaError_t launch_interchange(const FactorWork<T> &w, cudaStream_t s, bool marked = false);

template <typename T>
cudaError_t launch_trailing(const FactorWork<T> &w, int kmin, int mode, cudaStream_t s);

size_t tc_ops_floats(int n, int bmax);
// tcgen05 trailing update with split operands: TF32 (f16 = false) or scaled FP16 parts
cudaError_t launch_trailing_tc(const FactorWork<float> &w, float *ops, int kmin, bool f16, cudaStream_t s);

template <typename T>
cudaError_t launch_factor_init(const FactorWork<T> &w, cudaStream_t s);

// Deferred row interchanges of the L columns: record the permutation and bounds after panel
// `blk`; at the end permute the rows of every panel's L columns once.
template <typename T>
cudaError_t launch_panel_record(const FactorWork<T> &w, int blk, cudaStream_t s);
template <typename T>
cudaError_t launch_lrows_permute(const FactorWork<T> &w, int npanels, cudaStream_t s);

template <typename T>
cudaError_t launch_factor_finish(const FactorWork<T> &w, cudaStream_t s);

// Algorithm 2 stop at position k: the Schur complement counts as zero (lower triangle of
// A(k:n, k:n) and D(k:n) set to zero)
template <typename T>
cudaError_t launch_guard_zero(int n, int k, T *A, int lda, double *Dd, double *Ds, cudaStream_t s);

template <typename T>
int panel_max_grid(int d, int bw, int chunk_cap, int spec);

// Latency probe of the FP32 panel's per-step grid exchange (red.max of a key, grid barrier,
// read-back) on `grid` CTAs of the panel's size; bar and the key ring must be zero at launch.
int exchange_probe_grid();
cudaError_t launch_exchange_probe(unsigned *bar, unsigned long long *keys, int *status, int grid, int rounds,
                                  cudaStream_t s);
// Failure path of the bounded waits: a grid barrier that cannot complete on `grid` cooperative
// CTAs, each giving up after limit_ns (ST_TIMEOUT); CTA 0 writes its wait's duration
cudaError_t launch_wait_expiry(unsigned *bar, int *status, int grid, unsigned long long limit_ns,
                               unsigned long long *elapsed_ns, cudaStream_t s);

// Solves and refinement.  `work` holds solve_work_bytes<T>(n, nrhs) bytes.  reuse_inv: the
// inverted diagonal blocks (and FP32 couplings) in `work` are those of this L, n and nrhs from an
// earlier call (the solves of one refinement), so they are not recomputed.
template <typename T>
size_t solve_work_bytes(int n, int nrhs);
template <typename T>
cudaError_t launch_solve(int n, int nrhs, const T *L, int lda, const double *Dd, const double *Ds,
                         const int *perm, double *X, int ldx, T *work, int *flags, int *status,
                         const int *skip, cudaStream_t s, bool reuse_inv = false);

// One triangle of the solve (unit lower L, one right-hand side, iperm = identity): mode 0
// x <- L^{-1} x, mode 1 x <- L^{-T} x; work / flags as for launch_solve with nrhs = 1
template <typename T>
cudaError_t launch_tri_solve(int n, const T *L, int lda, const int *iperm, double *x, T *work, int *flags,
                             int *status, int mode, cudaStream_t s);
cudaError_t launch_iota(int n, int *p, cudaStream_t s);
// ||L||_1 (unit diagonal implied) as ordered bits of a non-negative double
template <typename T>
cudaError_t launch_l_norm1(int n, const T *L, int lda, unsigned long long *out, cudaStream_t s);

size_t symv_part_doubles(int n, int nrhs);
cudaError_t launch_symv_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                                 const double *Bv, int ldb, double *R, int ldr, double *part,
                                 unsigned long long *mx, const int *skip, cudaStream_t s);
cudaError_t launch_anorm(int n, const double *A, int lda, double *part, double *anorm, cudaStream_t s);
// berr from the residual maxima; conv = 1 when berr <= tol, 2 when a correction did not halve
// berr (stagnation or divergence; prev holds the previous berr, 0 before the first)
cudaError_t launch_refine_check(int nrhs, const unsigned long long *mx, const double *anorm, double tol, int *conv,
                                double *berr, double *prev, int *iters, int count_iter, cudaStream_t s);
cudaError_t launch_axpy_update(int n, int nrhs, double *X, int ldx, const double *D, int ldd,
                               const int *skip, cudaStream_t s);
// lower triangle of columns c0 .. c1-1 (c1 < 0: all) of an FP64 matrix, FP64 or rounded to FP32
cudaError_t launch_copy_lower_f64(int n, const double *src, int lds, void *dst, int ldd, int to_f32, cudaStream_t s,
                                  int c0 = 0, int c1 = -1);
// columns c0 .. c1-1 of B = Omega A (FP32); A must hold its final values in columns < c1
cudaError_t launch_sketch_cols_f32(int n, int d, const float *A, int lda, const float *om, float *B, float *part,
                                   size_t part_floats, int c0, int c1, cudaStream_t s);

// Krylov basis operations of GMRES-based refinement (FP64, basis column-major with ld ldv).
// out[c] = V(:, c)^T w for c < ncol (part: gm_part_doubles(n, ncol) doubles, deterministic);
// w += sign * V(:, 0:ncol) h (h on the device); w *= f.
size_t gm_part_doubles(int n, int ncol_max);
cudaError_t launch_gm_dots(int n, int ncol, const double *V, int ldv, const double *w, double *part, double *out,
                           cudaStream_t s);
cudaError_t launch_gm_update(int n, int ncol, const double *V, int ldv, const double *h, double sign, double *w,
                             cudaStream_t s);
cudaError_t launch_gm_scale(int n, double f, double *w, cudaStream_t s);

// Batched small systems (one CTA per system at a time).  info of a system that met a NaN or
// Inf is BT_INFO_NONFINITE.
constexpr int BT_INFO_NONFINITE = -4;
size_t batched_max_smem();
template <typename T>
size_t batched_factor_smem(int d, int b, int nmax);
template <typename TL>
size_t batched_refine_smem(int nrhs, int nmax);
// order: systems by decreasing n; above (nmax + 1 ints, may be NULL): above[v] = systems with n > v
cudaError_t launch_batched_order(int batch, int nmax, const int *n, int *order, int *above, cudaStream_t s);
size_t batched_factor_scratch_ints(int b, int nmax);   // per CTA
// resident CTAs of the factor kernel with nt (128, 256 or 512) threads per CTA (0: error)
template <typename T>
int batched_factor_grid(int d, int b, int nmax, int nt);
// one launch over order[*first .. *last) (NULL: 0 and batch) with nt threads per CTA
template <typename T>
cudaError_t launch_batched_factor(int batch, int d, int b, int nmax, const int *n, const double *const *A64,
                                  const int *lda64, T *const *A, const int *lda, double *const *Dd, double *const *Ds,
                                  int *const *perm, const T *om, double alpha, int *info, const int *order,
                                  int *ticket, int *pscr, int grid, int nt, const int *first, const int *last,
                                  cudaStream_t s);
template <typename TL>
cudaError_t launch_batched_refine(int batch, int nrhs, int nmax, int max_iter, double tol, const int *n,
                                  const TL *const *LA, const int *ldla, const double *const *Dd,
                                  const double *const *Ds, const int *const *perm, const double *const *A64,
                                  const int *lda64, const double *const *Bv, const int *ldb, double *const *X,
                                  const int *ldx, double *berr, int *iters, const int *order, int *ticket,
                                  cudaStream_t s);

}  // namespace rcpk

