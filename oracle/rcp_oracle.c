/*
 * rcp_oracle.c -- plain, slow, FP64 CPU oracle for randomized complete pivoting (RCP).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file; only the tests, the package smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant generator with the
 * CUDA library: the only thing both sides agree on is the published definition of
 * the Philox4x64-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), written here from that
 * definition.
 *
 * Every routine works on full (both triangles) column-major n x n FP64 arrays,
 * element (i, j) at a[i + j*n], and updates the Schur complement eagerly after every
 * pivot, i.e. Algorithm 1 of the paper with b = q = 1 (Section 3.1), so that a reader
 * can check each step against the paper.  There is no blocking, fusion or
 * reordering beyond what the paper states.
 *
 * Conventions shared with the tests (not with the GPU code):
 *   perm[i]  = original index of the row/column that ends at position i, so that
 *              A(perm[i], perm[j]) = (L D L^T)(i, j)          (Eq. for Pi^T A Pi = L D L^T)
 *   L        = n x n unit lower triangular (full array, explicit unit diagonal)
 *   Dd[i]    = D(i, i);  Ds[i] = D(i+1, i) (0 for a 1x1 block and for i = n-1)
 *   info     = 1 + position of the first exactly zero 1x1 pivot, 0 if none (LAPACK style)
 *
 * Readings of the paper where it is silent:
 *   - ties in every argmax go to the smallest current position;
 *   - the comparisons in the pivot rules are the non-strict ">=" printed in the figures;
 *   - SBKP case (0) (lambda = 0) takes a_kk as a 1x1 pivot with a zero multiplier
 *     column; if a_kk = 0 too, info records the position and the step continues;
 *   - SBKP case (3) with r = k+1 needs no interchange;
 *   - the q = b block sketch update uses L11^{-T} (derived from the update identity
 *     of Section 3; the printed formula shows L11^{-1}).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(a, n, i, j) ((a)[(size_t)(i) + (size_t)(j) * (size_t)(n)])

/* ------------------------------------------------------------------------------ */
/* Philox4x64-10 (SC'11).  Round: two 64x64->128 products of the even words with   */
/* the multipliers, the high halves xor-ed with the odd words and the key, then    */
/* the key is bumped by the Weyl constants.                                        */
/* ------------------------------------------------------------------------------ */
static void mul_hi_lo(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mul_hi_lo(M0, x0, &hi0, &lo0);
        mul_hi_lo(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Gaussian sketch matrix Omega (d x n, column-major, entries i.i.d. N(0,1)), the
 * random matrix drawn at the start of Algorithm 1.  Entry pair (2t, 2t+1) of column j
 * comes from one Philox call with counter (j, t, stream, 0) and key (seed, 0):
 *   u1 = (top 53 bits of w0 + 1) * 2^-53  in (0, 1],   u2 = (top 53 bits of w1) * 2^-53,
 *   rho = sqrt(-2 ln u1),  Omega(2t, j) = rho cos(2 pi u2),  Omega(2t+1, j) = rho sin(2 pi u2)
 * (Box and Muller, 1958).  Words w2, w3 are not used. */
void oracle_omega(uint64_t seed, uint64_t stream, int d, int n, double *om)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < n; ++j) {
        for (int t = 0; 2 * t < d; ++t) {
            uint64_t ctr[4] = {(uint64_t)j, (uint64_t)t, stream, 0};
            uint64_t key[2] = {seed, 0};
            uint64_t w[4];
            oracle_philox4x64_10(ctr, key, w);
            double u1 = ((double)(w[0] >> 11) + 1.0) * 0x1.0p-53;
            double u2 = (double)(w[1] >> 11) * 0x1.0p-53;
            double rho = sqrt(-2.0 * log(u1));
            double th = two_pi * u2;
            om[(size_t)(2 * t) + (size_t)j * d] = rho * cos(th);
            if (2 * t + 1 < d) om[(size_t)(2 * t + 1) + (size_t)j * d] = rho * sin(th);
        }
    }
}

/* B = Omega A (the random projection of Section 3), plain triple loop. */
void oracle_sketch(int n, int d, const double *om, const double *a, double *b)
{
    for (int j = 0; j < n; ++j)
        for (int r = 0; r < d; ++r) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += om[(size_t)r + (size_t)i * d] * AT(a, n, i, j);
            b[(size_t)r + (size_t)j * d] = s;
        }
}

/* ------------------------------------------------------------------------------ */
/* Symmetric interchange of positions p and q in every array the pivot touches:    */
/* rows and columns of the Schur-complement array A, columns of the sketch B,      */
/* rows of the already computed columns 0..k-1 of L, and the permutation record.   */
/* ------------------------------------------------------------------------------ */
static void swap_d(double *x, double *y) { double t = *x; *x = *y; *y = t; }

static void interchange(int n, int k, int p, int q, double *a, int d, double *b, double *l, int *perm)
{
    if (p == q) return;
    for (int j = 0; j < n; ++j) swap_d(&AT(a, n, p, j), &AT(a, n, q, j));   /* rows    */
    for (int i = 0; i < n; ++i) swap_d(&AT(a, n, i, p), &AT(a, n, i, q));   /* columns */
    if (b)
        for (int r = 0; r < d; ++r) swap_d(&b[(size_t)r + (size_t)p * d], &b[(size_t)r + (size_t)q * d]);
    for (int j = 0; j < k; ++j) swap_d(&AT(l, n, p, j), &AT(l, n, q, j));
    int t = perm[p]; perm[p] = perm[q]; perm[q] = t;
}

/* Largest |entry| of the trailing block A(k:n, k:n), used for rho_elem. */
static double trailing_maxabs(int n, int k, const double *a)
{
    double m = 0.0;
    for (int j = k; j < n; ++j)
        for (int i = k; i < n; ++i) if (fabs(AT(a, n, i, j)) > m) m = fabs(AT(a, n, i, j));
    return m;
}

/* One elimination step with an s x s pivot block at positions k..k+s-1 (already moved
 * there): D_k = A11, L21 = A21 A11^{-1}, Schur complement A22 -= A21 A11^{-1} A21^T
 * (Section 2.2).  The 2x2 inverse follows the scaled form used by LAPACK's SYTRF:
 * with e = a21, a = a11/e, c = a22/e, 1/(a c - 1) factors the determinant.  Returns the
 * zero-pivot flag (1x1 block with D = 0). */
static int eliminate(int n, int k, int s, double *a, double *l, double *dd, double *ds)
{
    int zero = 0;
    AT(l, n, k, k) = 1.0;
    if (s == 1) {
        double piv = AT(a, n, k, k);
        dd[k] = piv;
        ds[k] = 0.0;
        if (piv == 0.0) {
            zero = 1;
            for (int i = k + 1; i < n; ++i) AT(l, n, i, k) = 0.0;
        } else {
            for (int i = k + 1; i < n; ++i) AT(l, n, i, k) = AT(a, n, i, k) / piv;
        }
        for (int j = k + 1; j < n; ++j)
            for (int i = k + 1; i < n; ++i)
                AT(a, n, i, j) -= AT(l, n, i, k) * piv * AT(l, n, j, k);
    } else {
        double a11 = AT(a, n, k, k), a21 = AT(a, n, k + 1, k), a22 = AT(a, n, k + 1, k + 1);
        dd[k] = a11; dd[k + 1] = a22; ds[k] = a21; ds[k + 1] = 0.0;
        AT(l, n, k + 1, k + 1) = 1.0;
        AT(l, n, k + 1, k) = 0.0;
        /* [l_i1 l_i2] = [a_i1 a_i2] * inv([[a11, a21], [a21, a22]]) */
        double aa = a11 / a21, cc = a22 / a21, t = 1.0 / (aa * cc - 1.0);
        for (int i = k + 2; i < n; ++i) {
            double x1 = AT(a, n, i, k) / a21, x2 = AT(a, n, i, k + 1) / a21;
            AT(l, n, i, k) = t * (cc * x1 - x2);
            AT(l, n, i, k + 1) = t * (aa * x2 - x1);
        }
        /* A22 -= [a_i1 a_i2] * [l_j1 l_j2]^T  (= L D L^T restricted to the trailing block) */
        for (int j = k + 2; j < n; ++j)
            for (int i = k + 2; i < n; ++i)
                AT(a, n, i, j) -= AT(a, n, i, k) * AT(l, n, j, k) + AT(a, n, i, k + 1) * AT(l, n, j, k + 1);
    }
    /* the eliminated rows/columns of the Schur-complement array are no longer used */
    for (int t2 = k; t2 < k + s; ++t2)
        for (int i = 0; i < n; ++i) { if (i >= k + s) { AT(a, n, i, t2) = 0.0; AT(a, n, t2, i) = 0.0; } }
    return zero;
}

/* Per-step record for the tests. */
typedef struct {
    int k;          /* position of the step                                           */
    int pi;         /* sketch pivot: position chosen by the column-norm argmax        */
    int r;          /* SBKP r (position, after the sketch interchange), -1 if none    */
    int kase;       /* SBKP case 0..3                                                 */
    int s;          /* pivot size                                                     */
    double norm2;   /* ||B(:, pi)||_2^2                                                */
    double lambda;  /* SBKP lambda                                                    */
    /* margins of the step's decisions (diagnostics; no decision reads them):           */
    double norm2_next;  /* second largest ||B(:, j)||_2^2 over the candidates (-1: none) */
    double lam_next;    /* second largest |a_ik| over i > k (-1: none)                  */
    double akk;         /* |a_kk| compared with alpha lambda                            */
    double arr;         /* |a_rr| compared with alpha lambda (cases 2/3), else -1       */
} oracle_step;

/* Simplified Bunch-Kaufman pivoting (Figure "SBKP") on column k of the current
 * Schur complement.  Performs the interchange it prescribes and returns s. */
static int sbkp(int n, int k, double alpha, double *a, int d, double *b, double *l, int *perm,
                int *kase_out, int *r_out, double *lam_out, oracle_step *rec)
{
    double lam = 0.0;
    int r = -1;
    for (int i = k + 1; i < n; ++i)
        if (fabs(AT(a, n, i, k)) > lam) { lam = fabs(AT(a, n, i, k)); r = i; }
    *lam_out = lam;
    *r_out = r;
    rec->lam_next = -1.0;
    for (int i = k + 1; i < n; ++i)
        if (i != r && fabs(AT(a, n, i, k)) > rec->lam_next) rec->lam_next = fabs(AT(a, n, i, k));
    rec->akk = fabs(AT(a, n, k, k));
    rec->arr = r >= 0 ? fabs(AT(a, n, r, r)) : -1.0;
    if (lam == 0.0) { *kase_out = 0; return 1; }
    if (fabs(AT(a, n, k, k)) >= alpha * lam) { *kase_out = 1; return 1; }
    if (fabs(AT(a, n, r, r)) >= alpha * lam) {
        *kase_out = 2;
        interchange(n, k, k, r, a, d, b, l, perm);
        return 1;
    }
    *kase_out = 3;
    if (r != k + 1) interchange(n, k, k + 1, r, a, d, b, l, perm);
    return 2;
}

/* Sketch update after an s x s pivot at k (Eq. "Update matrix B", q = 1):
 * B(:, k+s:n) -= B(:, k:k+s-1) L(k+s:n, k:k+s-1)^T. */
static void sketch_update_rank_s(int n, int d, int k, int s, double *b, const double *l)
{
    for (int j = k + s; j < n; ++j)
        for (int t = k; t < k + s; ++t) {
            double ljt = AT(l, n, j, t);
            for (int r = 0; r < d; ++r) b[(size_t)r + (size_t)j * d] -= b[(size_t)r + (size_t)t * d] * ljt;
        }
}

/* b-step partial QR with column pivoting (Businger and Golub) of B(:, k:n), used by
 * Algorithm 1 with q = b to pick q candidate pivots at once.  Works on a copy of B with
 * Householder reflections; the residual column norms are recomputed from scratch at
 * every step.  Returns the chosen positions (as the interchanges are applied to the
 * real arrays right away, candidate t always sits at position k+t). */
static void partial_qrcp_select(int n, int d, int k, int q, double *a, double *b, double *l, int *perm)
{
    int m = n - k;
    double *w = (double *)malloc(sizeof(double) * (size_t)d * (size_t)m);
    for (int j = 0; j < m; ++j)
        for (int r = 0; r < d; ++r) w[(size_t)r + (size_t)j * d] = b[(size_t)r + (size_t)(k + j) * d];
    int steps = q < m ? q : m;
    if (steps > d) steps = d;
    for (int t = 0; t < steps; ++t) {
        int best = -1;
        double bn = -1.0;
        for (int j = t; j < m; ++j) {
            double s2 = 0.0;
            for (int r = t; r < d; ++r) s2 += w[(size_t)r + (size_t)j * d] * w[(size_t)r + (size_t)j * d];
            if (s2 > bn) { bn = s2; best = j; }
        }
        if (best != t) {
            for (int r = 0; r < d; ++r) swap_d(&w[(size_t)r + (size_t)t * d], &w[(size_t)r + (size_t)best * d]);
            interchange(n, k, k + t, k + best, a, d, b, l, perm);
        }
        /* Householder reflection zeroing w(t+1:d, t) */
        double nrm = 0.0;
        for (int r = t; r < d; ++r) nrm += w[(size_t)r + (size_t)t * d] * w[(size_t)r + (size_t)t * d];
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        double x0 = w[(size_t)t + (size_t)t * d];
        double alpha = x0 >= 0 ? -nrm : nrm;
        double *v = (double *)malloc(sizeof(double) * (size_t)d);
        for (int r = 0; r < d; ++r) v[r] = 0.0;
        v[t] = x0 - alpha;
        for (int r = t + 1; r < d; ++r) v[r] = w[(size_t)r + (size_t)t * d];
        double vv = 0.0;
        for (int r = t; r < d; ++r) vv += v[r] * v[r];
        if (vv > 0.0)
            for (int j = t; j < m; ++j) {
                double dot = 0.0;
                for (int r = t; r < d; ++r) dot += v[r] * w[(size_t)r + (size_t)j * d];
                double f = 2.0 * dot / vv;
                for (int r = t; r < d; ++r) w[(size_t)r + (size_t)j * d] -= f * v[r];
            }
        free(v);
    }
    free(w);
}

/*
 * RCP factorization, Algorithm 1 of the paper, run with an eager Schur complement.
 *   q_mode = 1 : one sketch pivot per step, B updated after every step (q = 1).
 *   q_mode = 2 : q = b, a b-step partial QRCP of B at the start of every block of b
 *                eliminated columns, and one block update of B at the end of the block.
 * a [n*n]     : in: symmetric A (both triangles); destroyed (Schur-complement workspace)
 * om [d*n]    : the Gaussian sketch matrix Omega
 * l [n*n], dd [n], ds [n], perm [n] : the factorization (conventions at the top)
 * steps       : optional per-step record (up to n entries), nsteps its count
 * snap_b, snap_a, snap_perm : optional snapshots (n x d*n, n x n*n, n x n) of B, of the
 *               Schur-complement array and of perm after each step (tiny n only; else NULL)
 * stats [4]   : rho_elem (max over all Schur complements / max|A|), number of 2x2
 *               blocks, min over steps of ||B(:,pi)|| / ||B||_{1,2}, max|L_ij| (i > j)
 * guard_r, guard_eps, seed, guard_out [2] : the safeguard of Algorithm 2 (q = 1 only;
 *               guard_r = 0: off).  With beta = ||B^(1)||_{1,2} and delta = (j + 1) / r after j
 *               recomputations of the sketch, the pivot of step k > 0 (already interchanged to
 *               position k, a symmetric permutation of the unfactored part) is accepted when its
 *               sketch column norm t >= eps^delta beta.  Otherwise, while j + 1 < r, a new
 *               Omega' (d x (n-k), Philox stream j + 1, columns indexed from position k) gives
 *               B(:, k:n) = Omega' S_k for the current Schur complement S_k, delta grows by 1/r
 *               and the argmax and interchange are taken again; if t is still below
 *               eps^delta beta (or no recomputation is left) the Schur complement counts as
 *               zero: the factorization stops with D(k:n, k:n) = 0, L(k:n, k:n) = I and
 *               info = k + 1.  guard_out = (rank k at the stop, or n; recomputations made).
 * Returns info.
 */
int oracle_rcp(int n, double *a, int d, const double *om, double alpha, int q_mode, int bsize,
               double *l, double *dd, double *ds, int *perm,
               oracle_step *steps, int *nsteps, double *snap_b, double *snap_a, int *snap_perm,
               double *stats, int guard_r, double guard_eps, uint64_t seed, int *guard_out)
{
    int info = 0, ns = 0, n2 = 0;
    double *b = (double *)malloc(sizeof(double) * (size_t)d * (size_t)(n > 0 ? n : 1));
    double amax = trailing_maxabs(n, 0, a), growth = amax;
    oracle_sketch(n, d, om, a, b);
    double beta = 0.0;
    for (int j = 0; j < n; ++j) {
        double s2 = 0.0;
        for (int r = 0; r < d; ++r) s2 += b[(size_t)r + (size_t)j * d] * b[(size_t)r + (size_t)j * d];
        if (s2 > beta) beta = s2;
    }
    double min_ratio = 1.0;
    memset(l, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; ++i) { perm[i] = i; dd[i] = 0.0; ds[i] = 0.0; }

    int k = 0;
    int blk_start = 0, blk_cols = 0, blk_len = 0;   /* q = b bookkeeping */
    int nresk = 0, stopped = 0;                      /* Algorithm 2 */
    while (k < n - 1) {
        oracle_step st;
        memset(&st, 0, sizeof st);
        st.k = k;
        if (q_mode == 1) {
            /* pi_k = argmax_{k <= j < n} ||B(:, j)||_2 (squared norms compared; ties to the
             * smallest position), then the interchange k <-> pi_k */
            int pi = k;
            double best = -1.0, second = -1.0;
            for (int j = k; j < n; ++j) {
                double s2 = 0.0;
                for (int r = 0; r < d; ++r) s2 += b[(size_t)r + (size_t)j * d] * b[(size_t)r + (size_t)j * d];
                if (s2 > best) { second = best; best = s2; pi = j; }
                else if (s2 > second) second = s2;
            }
            st.norm2_next = second;
            interchange(n, k, k, pi, a, d, b, l, perm);
            if (guard_r > 0 && k > 0) {
                /* Algorithm 2: t^2 against (eps^delta beta)^2 (beta holds ||B^(1)||_{1,2}^2) */
                double thr2 = beta * pow(guard_eps, 2.0 * (double)(nresk + 1) / (double)guard_r);
                if (best < thr2 && nresk + 1 < guard_r) {
                    ++nresk;
                    int m = n - k;
                    double *om2 = (double *)malloc(sizeof(double) * (size_t)d * (size_t)m);
                    oracle_omega(seed, (uint64_t)nresk, d, m, om2);
                    for (int jj = 0; jj < m; ++jj)
                        for (int r = 0; r < d; ++r) {
                            double v = 0.0;
                            for (int ii = 0; ii < m; ++ii) v += om2[(size_t)r + (size_t)ii * d] * AT(a, n, k + ii, k + jj);
                            b[(size_t)r + (size_t)(k + jj) * d] = v;
                        }
                    free(om2);
                    pi = k;
                    best = -1.0;
                    for (int j = k; j < n; ++j) {
                        double s2 = 0.0;
                        for (int r = 0; r < d; ++r) s2 += b[(size_t)r + (size_t)j * d] * b[(size_t)r + (size_t)j * d];
                        if (s2 > best) { best = s2; pi = j; }
                    }
                    interchange(n, k, k, pi, a, d, b, l, perm);
                    thr2 = beta * pow(guard_eps, 2.0 * (double)(nresk + 1) / (double)guard_r);
                }
                if (best < thr2) { stopped = 1; break; }
            }
            st.pi = pi;
            st.norm2 = best;
            if (beta > 0.0 && sqrt(best / beta) < min_ratio) min_ratio = sqrt(best / beta);
        } else if (blk_cols == 0) {
            /* first step of a block: b-step partial QRCP on B(:, k:n); the candidates are
             * interchanged to positions k..k+b-1 */
            blk_start = k;
            blk_len = bsize < n - k ? bsize : n - k;
            partial_qrcp_select(n, d, k, bsize, a, b, l, perm);
            st.pi = k;
        }
        int kase, r;
        double lam;
        int s = sbkp(n, k, alpha, a, d, b, l, perm, &kase, &r, &lam, &st);
        st.kase = kase; st.r = r; st.lambda = lam; st.s = s;
        if (eliminate(n, k, s, a, l, dd, ds) && info == 0) info = k + 1;
        if (s == 2) ++n2;
        double g = trailing_maxabs(n, k + s, a);
        if (g > growth) growth = g;
        if (q_mode == 1) {
            if (k + s < n) sketch_update_rank_s(n, d, k, s, b, l);
        } else {
            blk_cols += s;
            if (blk_cols >= blk_len) {
                /* end of the block: B(:, k1:n) -= B(:, blk) L11^{-T} L21^T, where B(:, blk)
                 * is the block-start sketch (with the block's interchanges applied) */
                int k0 = blk_start, k1 = k + s, m = k1 - k0;
                if (k1 < n) {
                    /* Y = B(:, blk) L11^{-T}, i.e. Y L11^T = B(:, blk), column by column */
                    double *y = (double *)malloc(sizeof(double) * (size_t)d * (size_t)m);
                    for (int c = 0; c < m; ++c)
                        for (int rr = 0; rr < d; ++rr) {
                            double v = b[(size_t)rr + (size_t)(k0 + c) * d];
                            for (int c2 = 0; c2 < c; ++c2) v -= y[(size_t)rr + (size_t)c2 * d] * AT(l, n, k0 + c, k0 + c2);
                            y[(size_t)rr + (size_t)c * d] = v;   /* L11 has a unit diagonal */
                        }
                    for (int j = k1; j < n; ++j)
                        for (int c = 0; c < m; ++c) {
                            double ljc = AT(l, n, j, k0 + c);
                            for (int rr = 0; rr < d; ++rr) b[(size_t)rr + (size_t)j * d] -= y[(size_t)rr + (size_t)c * d] * ljc;
                        }
                    free(y);
                }
                blk_cols = 0;
            }
        }
        if (steps) steps[ns] = st;
        if (snap_b) memcpy(snap_b + (size_t)ns * d * n, b, sizeof(double) * (size_t)d * n);
        if (snap_a) memcpy(snap_a + (size_t)ns * n * n, a, sizeof(double) * (size_t)n * n);
        if (snap_perm) memcpy(snap_perm + (size_t)ns * n, perm, sizeof(int) * (size_t)n);
        ++ns;
        k += s;
    }
    if (stopped) {
        /* Algorithm 2: the Schur complement of order n - k counts as zero */
        for (int i = k; i < n; ++i) {
            dd[i] = 0.0;
            ds[i] = 0.0;
            for (int j = k; j < n; ++j) AT(l, n, i, j) = i == j ? 1.0 : 0.0;
        }
        if (info == 0) info = k + 1;
    } else if (k == n - 1) {
        /* last position: D(n, n) = A(n, n) */
        dd[k] = AT(a, n, k, k);
        ds[k] = 0.0;
        AT(l, n, k, k) = 1.0;
        if (dd[k] == 0.0 && info == 0) info = k + 1;
    }
    free(b);
    if (guard_out) { guard_out[0] = stopped ? k : n; guard_out[1] = nresk; }
    if (nsteps) *nsteps = ns;
    if (stats) {
        double lmax = 0.0;
        for (int j = 0; j < n; ++j)
            for (int i = j + 1; i < n; ++i) if (fabs(AT(l, n, i, j)) > lmax) lmax = fabs(AT(l, n, i, j));
        stats[0] = amax > 0.0 ? growth / amax : 0.0;
        stats[1] = (double)n2;
        stats[2] = min_ratio;
        stats[3] = lmax;
    }
    return info;
}

/* ------------------------------------------------------------------------------ */
/* Comparison methods (oracle only).                                              */
/* ------------------------------------------------------------------------------ */

/* Bunch-Kaufman partial pivoting, Figure "BKPP": lambda and r from column k, sigma the
 * largest off-diagonal magnitude in column r, cases (0)-(4); ties to the smallest index. */
int oracle_bk(int n, double *a, double alpha, double *l, double *dd, double *ds, int *perm, double *stats)
{
    int info = 0, n2 = 0;
    double amax = trailing_maxabs(n, 0, a), growth = amax;
    memset(l, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; ++i) { perm[i] = i; dd[i] = 0.0; ds[i] = 0.0; }
    int k = 0;
    while (k < n - 1) {
        double lam = 0.0;
        int r = -1;
        for (int i = k + 1; i < n; ++i)
            if (fabs(AT(a, n, i, k)) > lam) { lam = fabs(AT(a, n, i, k)); r = i; }
        int s = 1;
        if (lam == 0.0) {
            s = 1;                                                  /* (0) */
        } else if (fabs(AT(a, n, k, k)) >= alpha * lam) {
            s = 1;                                                  /* (1) */
        } else {
            double sigma = 0.0;
            for (int i = k; i < n; ++i)
                if (i != r && fabs(AT(a, n, i, r)) > sigma) sigma = fabs(AT(a, n, i, r));
            if (fabs(AT(a, n, k, k)) * sigma >= alpha * lam * lam) {
                s = 1;                                              /* (2) */
            } else if (fabs(AT(a, n, r, r)) >= alpha * sigma) {
                s = 1;                                              /* (3) */
                interchange(n, k, k, r, a, 0, NULL, l, perm);
            } else {
                s = 2;                                              /* (4) */
                if (r != k + 1) interchange(n, k, k + 1, r, a, 0, NULL, l, perm);
            }
        }
        if (eliminate(n, k, s, a, l, dd, ds) && info == 0) info = k + 1;
        if (s == 2) ++n2;
        double g = trailing_maxabs(n, k + s, a);
        if (g > growth) growth = g;
        k += s;
    }
    if (k == n - 1) {
        dd[k] = AT(a, n, k, k);
        AT(l, n, k, k) = 1.0;
        if (dd[k] == 0.0 && info == 0) info = k + 1;
    }
    if (stats) { stats[0] = amax > 0.0 ? growth / amax : 0.0; stats[1] = (double)n2; }
    return info;
}

/* Bunch-Parlett complete diagonal pivoting (the textbook rule; the paper cites it
 * without pseudo-code): mu0 = largest off-diagonal magnitude of the whole Schur
 * complement at (p, q), p > q; mu1 = largest diagonal magnitude at position t.
 * If mu1 >= alpha mu0: 1x1 pivot, t moved to k.  Otherwise a 2x2 pivot, q moved to k and
 * p to k+1.  Ties to the smallest (column, then row) index. */
int oracle_bp(int n, double *a, double alpha, double *l, double *dd, double *ds, int *perm, double *stats)
{
    int info = 0, n2 = 0;
    double amax = trailing_maxabs(n, 0, a), growth = amax;
    memset(l, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; ++i) { perm[i] = i; dd[i] = 0.0; ds[i] = 0.0; }
    int k = 0;
    while (k < n - 1) {
        double mu0 = 0.0, mu1 = 0.0;
        int p0 = -1, q0 = -1, t = k;
        for (int j = k; j < n; ++j) {
            if (fabs(AT(a, n, j, j)) > mu1) { mu1 = fabs(AT(a, n, j, j)); t = j; }
            for (int i = j + 1; i < n; ++i)
                if (fabs(AT(a, n, i, j)) > mu0) { mu0 = fabs(AT(a, n, i, j)); p0 = i; q0 = j; }
        }
        int s;
        if (mu0 == 0.0 || mu1 >= alpha * mu0) {
            s = 1;
            interchange(n, k, k, t, a, 0, NULL, l, perm);
        } else {
            s = 2;
            /* move q0 to k, then p0 to k+1 (p0 > q0 >= k: the first swap leaves p0 in place) */
            interchange(n, k, k, q0, a, 0, NULL, l, perm);
            interchange(n, k, k + 1, p0, a, 0, NULL, l, perm);
        }
        if (eliminate(n, k, s, a, l, dd, ds) && info == 0) info = k + 1;
        if (s == 2) ++n2;
        double g = trailing_maxabs(n, k + s, a);
        if (g > growth) growth = g;
        k += s;
    }
    if (k == n - 1) {
        dd[k] = AT(a, n, k, k);
        AT(l, n, k, k) = 1.0;
        if (dd[k] == 0.0 && info == 0) info = k + 1;
    }
    if (stats) { stats[0] = amax > 0.0 ? growth / amax : 0.0; stats[1] = (double)n2; }
    return info;
}

/* ------------------------------------------------------------------------------ */
/* Solve and diagnostics.                                                          */
/* ------------------------------------------------------------------------------ */

/* Solution phase (Table "operation counts", solution row): with A(perm, perm) = L D L^T,
 * x(perm) = L^{-T} D^+ L^{-1} b(perm), D^+ the pseudo-inverse of D: a zero 1x1 block (an
 * exactly singular pivot, or the zero Schur complement where Algorithm 2 stopped) contributes
 * 0, which gives the basic solution of a rank-deficient factorization.  x [n*nrhs] holds b on
 * entry, x on exit. */
void oracle_ldlt_solve(int n, int nrhs, const double *l, const double *dd, const double *ds,
                       const int *perm, double *x)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int c = 0; c < nrhs; ++c) {
        double *xc = x + (size_t)c * n;
        for (int i = 0; i < n; ++i) y[i] = xc[perm[i]];
        for (int i = 0; i < n; ++i)                      /* L z = y (unit lower) */
            for (int j = 0; j < i; ++j) y[i] -= AT(l, n, i, j) * y[j];
        for (int i = 0; i < n; ++i) {                    /* D w = z */
            if (i + 1 < n && ds[i] != 0.0) {
                double a11 = dd[i], a21 = ds[i], a22 = dd[i + 1];
                double det = a11 * a22 - a21 * a21;
                double z1 = y[i], z2 = y[i + 1];
                y[i] = (a22 * z1 - a21 * z2) / det;
                y[i + 1] = (a11 * z2 - a21 * z1) / det;
                ++i;
            } else {
                y[i] = dd[i] != 0.0 ? y[i] / dd[i] : 0.0;
            }
        }
        for (int i = n - 1; i >= 0; --i)                 /* L^T v = w */
            for (int j = i + 1; j < n; ++j) y[i] -= AT(l, n, j, i) * y[j];
        for (int i = 0; i < n; ++i) xc[perm[i]] = y[i];
    }
    free(y);
}

/* Normwise relative backward error of Eq. "err": ||A x - b||_inf / (||A||_inf ||x||_inf),
 * the maximum over right-hand sides. */
double oracle_berr(int n, int nrhs, const double *a, const double *x, const double *rhs)
{
    double anorm = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += fabs(AT(a, n, i, j));
        if (s > anorm) anorm = s;
    }
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        const double *xc = x + (size_t)c * n, *bc = rhs + (size_t)c * n;
        double rn = 0.0, xn = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = bc[i];
            for (int j = 0; j < n; ++j) s -= AT(a, n, i, j) * xc[j];
            if (fabs(s) > rn) rn = fabs(s);
            if (fabs(xc[i]) > xn) xn = fabs(xc[i]);
        }
        double e = (anorm > 0.0 && xn > 0.0) ? rn / (anorm * xn) : (rn > 0.0 ? INFINITY : 0.0);
        if (e > worst) worst = e;
    }
    return worst;
}
