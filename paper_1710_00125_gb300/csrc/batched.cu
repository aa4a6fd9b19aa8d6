// batched.cu -- many independent small systems (n <= a few hundred): RCP factorization and
// FP64 iterative refinement, one persistent kernel per phase.
//
// Each CTA takes systems from an atomic ticket; the order puts the largest systems first
// (longest-processing-time-first scheduling), so the tail of the launch is made of small
// systems.  One CTA runs Algorithm 1 (q = 1) on one system, so every synchronization of the
// method is a CTA barrier, and the per-system state (sketch, panel) lives in shared memory:
//
//   Bs  d x nmax      the sketch B = Omega A, row-major ([r][j]), updated after every pivot
//   W   (b+1) x nmax  Schur-complement columns of the current panel ([t][j])
//   Lp  (b+1) x nmax  the panel's multipliers ([t][j])
//   c1, c2           the Schur columns k and r of the current step
//
// A itself (lower triangle, column-major) stays in global memory; row/column interchanges
// are applied to it at once, and the panel's trailing update A22 -= W Lp^T runs at the end of
// every panel.  The omega matrix is drawn once per call (d x nmax); system i uses its first n_i
// columns, which are the columns a d x n_i draw with the same seed gives.
#include <cfloat>
#include <climits>

#include "kernels.h"

namespace rcpk {

namespace bt {
constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int TILE = 32;          // sketch tiles
constexpr int MR = 16;            // sketch rows per thread: d <= 8 * MR = 128
constexpr unsigned FULLM = 0xffffffffu;
}  // namespace bt

// ---------------------------------------------------------------------------------------------
// block-wide argmax (value descending, index ascending), one barrier per call: the candidates
// go to one of two shared buffers, alternating between calls, and every thread reduces them.
// ---------------------------------------------------------------------------------------------
template <typename T>
struct BtCand {
    T v;
    int j;
};

template <typename T>
__device__ __forceinline__ bool bt_better(T v1, int j1, T v2, int j2) {
    return v1 > v2 || (v1 == v2 && j1 < j2);
}

template <typename T>
__device__ __forceinline__ BtCand<T> bt_argmax(BtCand<T> c, BtCand<T> (*red)[bt::WARPS], int &buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const T v = __shfl_xor_sync(bt::FULLM, c.v, off);
        const int j = __shfl_xor_sync(bt::FULLM, c.j, off);
        if (bt_better(v, j, c.v, c.j)) { c.v = v; c.j = j; }
    }
    if (lane == 0) red[buf][warp] = c;
    __syncthreads();
    BtCand<T> r = red[buf][0];
#pragma unroll
    for (int w2 = 1; w2 < bt::WARPS; ++w2) {
        const BtCand<T> x = red[buf][w2];
        if (bt_better(x.v, x.j, r.v, r.j)) r = x;
    }
    buf ^= 1;
    return r;
}

template <typename T>
__device__ __forceinline__ T bt_abs(T x) { return x < T(0) ? -x : x; }

template <typename T>
__device__ __forceinline__ T a_sym(const T *A, int lda, int i, int j) {
    return i >= j ? A[(size_t)i + (size_t)j * lda] : A[(size_t)j + (size_t)i * lda];
}

// Symmetric interchange of positions p != q in lower storage, all n rows and columns.
template <typename T>
__device__ void bt_sym_swap(T *A, int lda, int n, int p, int q) {
    if (p > q) { const int t = p; p = q; q = t; }
    for (int x = threadIdx.x; x < n; x += bt::THREADS) {
        T *u, *v;
        if (x < p) { u = A + (size_t)p + (size_t)x * lda; v = A + (size_t)q + (size_t)x * lda; }
        else if (x == p) { u = A + (size_t)p + (size_t)p * lda; v = A + (size_t)q + (size_t)q * lda; }
        else if (x < q) { u = A + (size_t)x + (size_t)p * lda; v = A + (size_t)q + (size_t)x * lda; }
        else if (x > q) { u = A + (size_t)x + (size_t)p * lda; v = A + (size_t)x + (size_t)q * lda; }
        else continue;
        const T t = *u; *u = *v; *v = t;
    }
}

// ---------------------------------------------------------------------------------------------
// factor kernel
// ---------------------------------------------------------------------------------------------
template <typename T>
struct BtFactorArgs {
    int batch, d, b, nmax;
    const int *n;
    const double *const *A64;   // optional FP64 source copied into A first (lower triangle)
    const int *lda64;
    T *const *A;
    const int *lda;
    double *const *Dd;
    double *const *Ds;
    int *const *perm;
    const T *om;                // d x nmax, column-major (ld d)
    double alpha;
    int *info;                  // [batch]
    const int *order;           // processing order (largest first)
    int *ticket;
};

// shared-memory elements of type T for one system of order <= nmax
__host__ __device__ inline size_t bt_factor_elems(int d, int b, int nmax) {
    const size_t panel = 2 * (size_t)(b + 1) * nmax;
    const size_t sk = (size_t)(bt::TILE + d) * (bt::TILE + 1);
    return (size_t)d * nmax + (panel > sk ? panel : sk) + 2 * (size_t)nmax + 2 * (size_t)d;
}

template <typename T>
size_t batched_factor_smem(int d, int b, int nmax) {
    return bt_factor_elems(d, b, nmax) * sizeof(T);
}

template <typename T>
__device__ void bt_factor_one(const BtFactorArgs<T> &a, int sys, T *sm, BtCand<T> (*red)[bt::WARPS], int &rbuf) {
    const int n = a.n[sys], d = a.d, nmax = a.nmax, tid = threadIdx.x;
    const int lda = a.lda[sys];
    T *A = a.A[sys];
    double *Dd = a.Dd[sys], *Ds = a.Ds[sys];
    int *perm = a.perm[sys];
    if (n <= 0) {
        if (tid == 0) a.info[sys] = 0;
        return;
    }
    const size_t panel = 2 * (size_t)(a.b + 1) * nmax;
    const size_t skel = (size_t)(bt::TILE + d) * (bt::TILE + 1);
    T *Bs = sm;                                        // [d][nmax]
    T *W = Bs + (size_t)d * nmax;                      // [b+1][nmax]
    T *Lp = W + (size_t)(a.b + 1) * nmax;              // [b+1][nmax]
    T *c1 = Bs + (size_t)d * nmax + (panel > skel ? panel : skel);
    T *c2 = c1 + nmax;
    T *pb = c2 + nmax;                                 // pivot sketch columns [2][d]

    // ---- optional FP64 source: copy the lower triangle into the factor array ----
    if (a.A64) {
        const double *S = a.A64[sys];
        const int lds = a.lda64[sys];
        for (int e = tid; e < n * n; e += bt::THREADS) {
            const int i = e % n, j = e / n;
            if (i >= j) A[(size_t)i + (size_t)j * lda] = (T)S[(size_t)i + (size_t)j * lds];
        }
    }
    for (int x = tid; x < n; x += bt::THREADS) perm[x] = x;
    __syncthreads();

    // ---- B = Omega(:, 0:n) A by 32 x 32 tiles of A (the sketch region aliases the panels) ----
    {
        T *As = W;                                     // [32][33]: As[i][j] = A_sym(i0 + i, j0 + j)
        T *Os = W + bt::TILE * (bt::TILE + 1);         // [d][33]:  Os[r][i] = Omega(r, i0 + i)
        const int jj = tid & 31, r0 = tid >> 5;
        for (int j0 = 0; j0 < n; j0 += bt::TILE) {
            T acc[bt::MR];
#pragma unroll
            for (int m = 0; m < bt::MR; ++m) acc[m] = T(0);
            for (int i0 = 0; i0 < n; i0 += bt::TILE) {
                for (int e = tid; e < bt::TILE * bt::TILE; e += bt::THREADS) {
                    const int lo = e & 31, hi = e >> 5;
                    if (i0 > j0) {          // A(i0 + lo, j0 + hi): column j0 + hi, coalesced
                        const int i = i0 + lo, j = j0 + hi;
                        As[lo * (bt::TILE + 1) + hi] = (i < n && j < n) ? A[(size_t)i + (size_t)j * lda] : T(0);
                    } else if (i0 < j0) {   // A(j0 + lo, i0 + hi) = A_sym(i0 + hi, j0 + lo)
                        const int i = i0 + hi, j = j0 + lo;
                        As[hi * (bt::TILE + 1) + lo] = (i < n && j < n) ? A[(size_t)j + (size_t)i * lda] : T(0);
                    } else {
                        const int i = i0 + lo, j = j0 + hi;
                        As[lo * (bt::TILE + 1) + hi] = (i < n && j < n) ? a_sym(A, lda, i, j) : T(0);
                    }
                }
                for (int e = tid; e < d * bt::TILE; e += bt::THREADS) {
                    const int r = e % d, i = e / d;
                    Os[r * (bt::TILE + 1) + i] = (i0 + i < n) ? a.om[(size_t)r + (size_t)(i0 + i) * d] : T(0);
                }
                __syncthreads();
#pragma unroll 4
                for (int i = 0; i < bt::TILE; ++i) {
                    const T av = As[i * (bt::TILE + 1) + jj];
#pragma unroll
                    for (int m = 0; m < bt::MR; ++m) {
                        const int r = r0 + 8 * m;
                        if (r < d) acc[m] += Os[r * (bt::TILE + 1) + i] * av;
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int m = 0; m < bt::MR; ++m) {
                const int r = r0 + 8 * m;
                if (r < d && j0 + jj < n) Bs[(size_t)r * nmax + j0 + jj] = acc[m];
            }
        }
    }
    __syncthreads();

    // ---- first pivot candidate: max column norm of B ----
    BtCand<T> cand{T(-1), INT_MAX};
    for (int j = tid; j < n; j += bt::THREADS) {
        T s = T(0);
        for (int r = 0; r < d; ++r) { const T v = Bs[(size_t)r * nmax + j]; s += v * v; }
        if (bt_better(s, j, cand.v, cand.j)) cand = BtCand<T>{s, j};
    }
    cand = bt_argmax(cand, red, rbuf);

    int info = 0, k = 0;
    bool bad = false;
    while (k < n && !bad) {
        const int k0 = k;
        int i = 0;
        while (i < a.b && k < n) {
            const int P = cand.j;
            if (P < k || P >= n || !isfinite((double)cand.v)) { bad = true; break; }
            const T *LpP = Lp + P;   // multipliers of the pivot row (old position P), stride nmax
            // ---- phase A: interchange k <-> P in A and the Schur column k (new labels) ----
            BtCand<T> lc{T(-1), INT_MAX};
            for (int x = tid; x < n; x += bt::THREADS) {
                if (x < k) {
                    if (P != k) {
                        T *u = A + (size_t)k + (size_t)x * lda, *v = A + (size_t)P + (size_t)x * lda;
                        const T t = *u; *u = *v; *v = t;
                    }
                    continue;
                }
                T av;
                int sx;            // old position of the row now at x
                if (x == k) {
                    av = A[(size_t)P + (size_t)P * lda];
                    if (P != k) A[(size_t)P + (size_t)P * lda] = A[(size_t)k + (size_t)k * lda];
                    A[(size_t)k + (size_t)k * lda] = av;
                    sx = P;
                } else if (x == P) {
                    av = A[(size_t)P + (size_t)k * lda];
                    sx = k;
                } else if (x < P) {
                    T *u = A + (size_t)x + (size_t)k * lda, *v = A + (size_t)P + (size_t)x * lda;
                    av = *v;
                    *v = *u;
                    *u = av;
                    sx = x;
                } else {
                    T *u = A + (size_t)x + (size_t)k * lda, *v = A + (size_t)x + (size_t)P * lda;
                    av = *v;
                    if (P != k) { *v = *u; *u = av; }
                    sx = x;
                }
                for (int t = 0; t < i; ++t) av -= W[(size_t)t * nmax + sx] * LpP[(size_t)t * nmax];
                c1[x] = av;
                if (x > k && bt_better(bt_abs(av), x, lc.v, lc.j)) lc = BtCand<T>{bt_abs(av), x};
            }
            for (int r = tid; r < d; r += bt::THREADS) pb[r] = Bs[(size_t)r * nmax + P];
            lc = bt_argmax(lc, red, rbuf);
            // ---- SBKP decision (every thread, from shared values) ----
            const int R = lc.j < n ? lc.j : -1;
            const double lam = R >= 0 ? (double)lc.v : 0.0;
            const double akk = (double)c1[k];
            if (!isfinite(lam) || !isfinite(akk)) { bad = true; break; }
            int kase;
            if (R < 0 || lam == 0.0) kase = 0;
            else if (fabs(akk) >= a.alpha * lam) kase = 1;
            else kase = 4;
            int s = 1, pswap = (P != k) ? P : -1;    // new position P still holds old column k of Bs
            const T *cp = c1;
            if (kase == 4) {
                // settle the k <-> P interchange in shared memory, then column R of the Schur complement
                if (P != k) {
                    for (int e = tid; e < d + 2 * i; e += bt::THREADS) {
                        T *u, *v;
                        if (e < d) { u = Bs + (size_t)e * nmax + k; v = Bs + (size_t)e * nmax + P; }
                        else if (e < d + i) { u = W + (size_t)(e - d) * nmax + k; v = W + (size_t)(e - d) * nmax + P; }
                        else { u = Lp + (size_t)(e - d - i) * nmax + k; v = Lp + (size_t)(e - d - i) * nmax + P; }
                        const T t = *u; *u = *v; *v = t;
                    }
                    if (tid == 0) { const int t = perm[k]; perm[k] = perm[P]; perm[P] = t; }
                }
                pswap = -1;
                __syncthreads();
                for (int x = k + tid; x < n; x += bt::THREADS) {
                    T av = a_sym(A, lda, x, R);
                    for (int t = 0; t < i; ++t) av -= W[(size_t)t * nmax + x] * Lp[(size_t)t * nmax + R];
                    c2[x] = av;
                }
                __syncthreads();
                const double arr = (double)c2[R];
                if (!isfinite(arr)) { bad = true; break; }
                kase = fabs(arr) >= a.alpha * lam ? 2 : 3;
                const int tgt = kase == 2 ? k : k + 1;
                if (R != tgt) {
                    bt_sym_swap(A, lda, n, tgt, R);
                    for (int e = tid; e < d + 2 * i; e += bt::THREADS) {
                        T *u, *v;
                        if (e < d) { u = Bs + (size_t)e * nmax + tgt; v = Bs + (size_t)e * nmax + R; }
                        else if (e < d + i) { u = W + (size_t)(e - d) * nmax + tgt; v = W + (size_t)(e - d) * nmax + R; }
                        else { u = Lp + (size_t)(e - d - i) * nmax + tgt; v = Lp + (size_t)(e - d - i) * nmax + R; }
                        const T t = *u; *u = *v; *v = t;
                    }
                    if (tid == 0) {
                        const int t = perm[tgt]; perm[tgt] = perm[R]; perm[R] = t;
                        T x = c1[tgt]; c1[tgt] = c1[R]; c1[R] = x;
                        x = c2[tgt]; c2[tgt] = c2[R]; c2[R] = x;
                    }
                }
                __syncthreads();
                for (int r = tid; r < d; r += bt::THREADS) {
                    pb[r] = Bs[(size_t)r * nmax + k];
                    if (k + 1 < n) pb[d + r] = Bs[(size_t)r * nmax + k + 1];
                }
                __syncthreads();
                if (kase == 2) cp = c2;
                else s = 2;
            } else if (P != k) {
                // 1x1 fast path: the k <-> P moves of the panel rows go with phase B
                for (int e = tid; e < 2 * i; e += bt::THREADS) {
                    T *u, *v;
                    if (e < i) { u = W + (size_t)e * nmax + k; v = W + (size_t)e * nmax + P; }
                    else { u = Lp + (size_t)(e - i) * nmax + k; v = Lp + (size_t)(e - i) * nmax + P; }
                    const T t = *u; *u = *v; *v = t;
                }
                if (tid == 0) { const int t = perm[k]; perm[k] = perm[P]; perm[P] = t; }
            }
            // ---- D block and multiplier scalars (FP64) ----
            double dp = 0.0, sa = 0.0, sc = 0.0, st = 0.0, sr = 0.0;
            if (s == 1) {
                dp = (double)cp[k];
                if (tid == 0) {
                    Dd[k] = dp;
                    Ds[k] = 0.0;
                }
                if (dp == 0.0 && info == 0) info = k + 1;
                dp = dp != 0.0 ? 1.0 / dp : 0.0;
            } else {
                const double a11 = (double)c1[k], a21 = (double)c1[k + 1], a22 = (double)c2[k + 1];
                sr = 1.0 / a21;
                sa = a11 * sr;
                sc = a22 * sr;
                st = 1.0 / (sa * sc - 1.0);
                if (tid == 0) {
                    Dd[k] = a11; Ds[k] = a21; Dd[k + 1] = a22; Ds[k + 1] = 0.0;
                }
            }
            // ---- phase B: multipliers, panel columns, rank-s sketch update and column norms ----
            BtCand<T> nc{T(-1), INT_MAX};
            const T finv = (T)dp, fa = (T)sa, fc = (T)sc, ft = (T)st, fr = (T)sr;
            for (int j = k + s + tid; j < n; j += bt::THREADS) {
                const int src = (j == pswap) ? k : j;
                T nrm = T(0);
                if (s == 1) {
                    const T cj = cp[j], l1 = cj * finv;
                    W[(size_t)i * nmax + j] = cj;
                    Lp[(size_t)i * nmax + j] = l1;
                    for (int r = 0; r < d; ++r) {
                        const T v = Bs[(size_t)r * nmax + src] - pb[r] * l1;
                        Bs[(size_t)r * nmax + j] = v;
                        nrm += v * v;
                    }
                } else {
                    const T x1 = c1[j] * fr, x2 = c2[j] * fr;
                    const T l1 = ft * (fc * x1 - x2), l2 = ft * (fa * x2 - x1);
                    W[(size_t)i * nmax + j] = c1[j];
                    W[(size_t)(i + 1) * nmax + j] = c2[j];
                    Lp[(size_t)i * nmax + j] = l1;
                    Lp[(size_t)(i + 1) * nmax + j] = l2;
                    for (int r = 0; r < d; ++r) {
                        T v = Bs[(size_t)r * nmax + j] - pb[r] * l1;
                        v -= pb[d + r] * l2;
                        Bs[(size_t)r * nmax + j] = v;
                        nrm += v * v;
                    }
                }
                if (bt_better(nrm, j, nc.v, nc.j)) nc = BtCand<T>{nrm, j};
            }
            if (s == 2 && tid == 0) Lp[(size_t)i * nmax + k + 1] = T(0);   // L(k+1, k) of a 2x2 block
            cand = bt_argmax(nc, red, rbuf);
            k += s;
            i += s;
        }
        if (bad) break;
        // ---- end of the panel: multipliers into A, then A22 -= W Lp^T (lower triangle) ----
        for (int e = tid; e < i * (n - k0); e += bt::THREADS) {
            const int t = e / (n - k0), p = k0 + e % (n - k0);
            if (p > k0 + t) A[(size_t)p + (size_t)(k0 + t) * lda] = Lp[(size_t)t * nmax + p];
        }
        const int m = n - k;
        if (m > 0) {
            const int nt = (m + 3) >> 2;
            for (int tt = tid; tt < nt * nt; tt += bt::THREADS) {
                const int I = tt % nt, J = tt / nt;
                if (I < J) continue;
                const int p0 = k + 4 * I, q0 = k + 4 * J;
                T acc[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
                for (int t = 0; t < i; ++t) {
                    T wv[4], lv[4];
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        wv[x] = p0 + x < n ? W[(size_t)t * nmax + p0 + x] : T(0);
                        lv[x] = q0 + x < n ? Lp[(size_t)t * nmax + q0 + x] : T(0);
                    }
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] += wv[x] * lv[y];
                }
#pragma unroll
                for (int y = 0; y < 4; ++y)
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const int p = p0 + x, q = q0 + y;
                        if (p < n && q < n && p >= q) A[(size_t)p + (size_t)q * lda] -= acc[x][y];
                    }
            }
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) a.info[sys] = BT_INFO_NONFINITE;
        __syncthreads();
        return;
    }
    for (int x = tid; x < n; x += bt::THREADS) A[(size_t)x + (size_t)x * lda] = (T)Dd[x];
    if (tid == 0) a.info[sys] = info;
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(bt::THREADS, 1) batched_factor_kernel(BtFactorArgs<T> a) {
    extern __shared__ __align__(16) unsigned char bt_raw[];
    __shared__ BtCand<T> red[2][bt::WARPS];
    __shared__ int s_idx;
    int rbuf = 0;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(a.ticket, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= a.batch) return;
        bt_factor_one<T>(a, a.order[idx], reinterpret_cast<T *>(bt_raw), red, rbuf);
    }
}

// ---------------------------------------------------------------------------------------------
// solve + FP64 refinement kernel
// ---------------------------------------------------------------------------------------------
template <typename TL>
struct BtRefineArgs {
    int batch, nrhs, nmax, max_iter;
    double tol;
    const int *n;
    const TL *const *LA;
    const int *ldla;
    const double *const *Dd;
    const double *const *Ds;
    const int *const *perm;
    const double *const *A64;   // NULL: solve only
    const int *lda64;
    const double *const *Bv;
    const int *ldb;
    double *const *X;
    const int *ldx;
    double *berr;               // [batch] (may be NULL)
    int *iters;                 // [batch] (may be NULL)
    const int *order;
    int *ticket;
};

constexpr int BT_RC = 16;       // right-hand sides per pass

template <typename TL>
size_t batched_refine_smem(int nrhs, int nmax) {
    const size_t rc = nrhs < BT_RC ? nrhs : BT_RC;
    return (rc * nmax * sizeof(TL) + 15) / 16 * 16 + 2 * rc * nmax * sizeof(double) + 2 * rc * sizeof(double);
}

// y <- (P L D L^T P^T)^{-1} y for the rc columns of y (shared, [c][nmax]); tmp is FP64 scratch.
template <typename TL>
__device__ void bt_solve(int n, int rc, int nmax, const TL *L, int lda, const double *Dd, const double *Ds,
                         const int *perm, TL *y, double *tmp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // perm comes from the factor kernel; an index outside [0, n) (a factor that never ran)
    // is replaced so that no access leaves the system's rows
    for (int e = tid; e < n * rc; e += bt::THREADS) {
        const int i = e % n, c = e / n;
        const int p = (unsigned)perm[i] < (unsigned)n ? perm[i] : i;
        tmp[(size_t)c * nmax + i] = (double)y[(size_t)c * nmax + p];
    }
    __syncthreads();
    for (int e = tid; e < n * rc; e += bt::THREADS) {
        const int i = e % n, c = e / n;
        y[(size_t)c * nmax + i] = (TL)tmp[(size_t)c * nmax + i];
    }
    __syncthreads();
    // forward, unit lower: 32-row diagonal blocks by one warp per column, then the rows below
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int nb = min(32, n - j0);
        for (int c = warp; c < rc; c += bt::WARPS) {
            TL *yc = y + (size_t)c * nmax;
            TL v = lane < nb ? yc[j0 + lane] : TL(0);
            for (int jj = 0; jj < nb - 1; ++jj) {
                const TL z = __shfl_sync(bt::FULLM, v, jj);
                if (lane > jj && lane < nb) v -= L[(size_t)(j0 + lane) + (size_t)(j0 + jj) * lda] * z;
            }
            if (lane < nb) yc[j0 + lane] = v;
        }
        __syncthreads();
        const int rows = n - j0 - nb;
        for (int e = tid; e < rows * rc; e += bt::THREADS) {
            const int r = j0 + nb + e % rows, c = e / rows;
            TL *yc = y + (size_t)c * nmax;
            TL sum = yc[r];
            for (int jj = 0; jj < nb; ++jj) sum -= L[(size_t)r + (size_t)(j0 + jj) * lda] * yc[j0 + jj];
            yc[r] = sum;
        }
        __syncthreads();
    }
    // block diagonal D: scaled 2x2 inverse in FP64
    for (int e = tid; e < n * rc; e += bt::THREADS) {
        const int i = e % n, c = e / n;
        TL *yc = y + (size_t)c * nmax;
        if (i > 0 && Ds[i - 1] != 0.0) continue;
        if (i + 1 < n && Ds[i] != 0.0) {
            const double bb = Ds[i], aa = Dd[i] / bb, cc = Dd[i + 1] / bb, den = aa * cc - 1.0;
            const double y1 = (double)yc[i] / bb, y2 = (double)yc[i + 1] / bb;
            yc[i] = (TL)((cc * y1 - y2) / den);
            yc[i + 1] = (TL)((aa * y2 - y1) / den);
        } else {
            yc[i] = (TL)((double)yc[i] / Dd[i]);
        }
    }
    __syncthreads();
    // backward with L^T, blocks from the bottom
    for (int jend = n; jend > 0; jend -= 32) {
        const int j0 = max(0, jend - 32), nb = jend - j0;
        for (int e = tid; e < nb * rc; e += bt::THREADS) {
            const int r = j0 + e % nb, c = e / nb;
            TL *yc = y + (size_t)c * nmax;
            TL sum = yc[r];
            for (int ii = jend; ii < n; ++ii) sum -= L[(size_t)ii + (size_t)r * lda] * yc[ii];
            yc[r] = sum;
        }
        __syncthreads();
        for (int c = warp; c < rc; c += bt::WARPS) {
            TL *yc = y + (size_t)c * nmax;
            TL v = lane < nb ? yc[j0 + lane] : TL(0);
            for (int jj = nb - 1; jj > 0; --jj) {
                const TL z = __shfl_sync(bt::FULLM, v, jj);
                if (lane < jj) v -= L[(size_t)(j0 + jj) + (size_t)(j0 + lane) * lda] * z;
            }
            if (lane < nb) yc[j0 + lane] = v;
        }
        __syncthreads();
    }
    for (int e = tid; e < n * rc; e += bt::THREADS) {
        const int i = e % n, c = e / n;
        const int p = (unsigned)perm[i] < (unsigned)n ? perm[i] : i;
        tmp[(size_t)c * nmax + p] = (double)y[(size_t)c * nmax + i];
    }
    __syncthreads();
    for (int e = tid; e < n * rc; e += bt::THREADS) {
        const int i = e % n, c = e / n;
        y[(size_t)c * nmax + i] = (TL)tmp[(size_t)c * nmax + i];
    }
    __syncthreads();
}

// r = b - A x (FP64) for the rows of this thread, RG right-hand sides per task
template <int RG>
__device__ void bt_residual(int n, int rc, int nmax, const double *A, int lda, const double *Bv, int ldb, int c0,
                            const double *x, double *r, double *rmax, double *xmax) {
    const int groups = rc / RG;
    for (int task = threadIdx.x; task < n * groups; task += bt::THREADS) {
        const int row = task % n, g = task / n;
        double acc[RG];
#pragma unroll
        for (int q = 0; q < RG; ++q) acc[q] = Bv[(size_t)row + (size_t)(c0 + g * RG + q) * ldb];
        const double *xg = x + (size_t)g * RG * nmax;
        for (int j = 0; j < n; ++j) {
            const double av = j <= row ? A[(size_t)row + (size_t)j * lda] : A[(size_t)j + (size_t)row * lda];
#pragma unroll
            for (int q = 0; q < RG; ++q) acc[q] -= av * xg[(size_t)q * nmax + j];
        }
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const int c = g * RG + q;
            r[(size_t)c * nmax + row] = acc[q];
            atomicMax(reinterpret_cast<unsigned long long *>(rmax + c), (unsigned long long)__double_as_longlong(fabs(acc[q])));
            atomicMax(reinterpret_cast<unsigned long long *>(xmax + c),
                      (unsigned long long)__double_as_longlong(fabs(xg[(size_t)q * nmax + row])));
        }
    }
}

template <typename TL>
__device__ void bt_refine_one(const BtRefineArgs<TL> &a, int sys, unsigned char *raw, double *s_an) {
    const int n = a.n[sys], nmax = a.nmax, tid = threadIdx.x;
    const int rcmax = a.nrhs < BT_RC ? a.nrhs : BT_RC;
    TL *y = reinterpret_cast<TL *>(raw);
    double *x = reinterpret_cast<double *>(raw + ((size_t)rcmax * nmax * sizeof(TL) + 15) / 16 * 16);
    double *tmp = x + (size_t)rcmax * nmax;
    double *rmax = tmp + (size_t)rcmax * nmax;
    double *xmax = rmax + rcmax;
    if (n <= 0) {
        if (tid == 0) {
            if (a.berr) a.berr[sys] = 0.0;
            if (a.iters) a.iters[sys] = 0;
        }
        return;
    }
    const TL *L = a.LA[sys];
    const int ldl = a.ldla[sys], ldb = a.ldb[sys], ldx = a.ldx[sys];
    const double *Bv = a.Bv[sys];
    double *X = a.X[sys];
    const double *A64 = a.A64 ? a.A64[sys] : nullptr;
    const int lda64 = a.A64 ? a.lda64[sys] : 0;
    // ||A||_inf of the symmetric matrix (lower storage)
    if (A64) {
        if (tid == 0) *s_an = 0.0;
        __syncthreads();
        for (int row = tid; row < n; row += bt::THREADS) {
            double sum = 0.0;
            for (int j = 0; j < n; ++j)
                sum += fabs(j <= row ? A64[(size_t)row + (size_t)j * lda64] : A64[(size_t)j + (size_t)row * lda64]);
            atomicMax(reinterpret_cast<unsigned long long *>(s_an), (unsigned long long)__double_as_longlong(sum));
        }
        __syncthreads();
    }
    const double an = A64 ? *s_an : 0.0;
    double worst = 0.0;
    int most = 0;
    for (int c0 = 0; c0 < a.nrhs; c0 += BT_RC) {
        const int rc = min(BT_RC, a.nrhs - c0);
        for (int e = tid; e < n * rc; e += bt::THREADS) {
            const int i = e % n, c = e / n;
            y[(size_t)c * nmax + i] = (TL)Bv[(size_t)i + (size_t)(c0 + c) * ldb];
        }
        __syncthreads();
        bt_solve<TL>(n, rc, nmax, L, ldl, a.Dd[sys], a.Ds[sys], a.perm[sys], y, tmp);
        for (int e = tid; e < n * rc; e += bt::THREADS) {
            const int i = e % n, c = e / n;
            x[(size_t)c * nmax + i] = (double)y[(size_t)c * nmax + i];
        }
        __syncthreads();
        int it = 0;
        double be = 0.0;
        while (A64) {
            for (int c = tid; c < rc; c += bt::THREADS) { rmax[c] = 0.0; xmax[c] = 0.0; }
            __syncthreads();
            // rows x groups of right-hand sides: enough tasks for the CTA even for small n
            int rg = rc;
            while (rg > 1 && n * (rc / rg) < bt::THREADS && (rg & 1) == 0) rg >>= 1;
            if (rg != 16 && rg != 8 && rg != 4 && rg != 2) rg = 1;
            switch (rg) {
                case 16: bt_residual<16>(n, rc, nmax, A64, lda64, Bv, ldb, c0, x, tmp, rmax, xmax); break;
                case 8: bt_residual<8>(n, rc, nmax, A64, lda64, Bv, ldb, c0, x, tmp, rmax, xmax); break;
                case 4: bt_residual<4>(n, rc, nmax, A64, lda64, Bv, ldb, c0, x, tmp, rmax, xmax); break;
                case 2: bt_residual<2>(n, rc, nmax, A64, lda64, Bv, ldb, c0, x, tmp, rmax, xmax); break;
                default: bt_residual<1>(n, rc, nmax, A64, lda64, Bv, ldb, c0, x, tmp, rmax, xmax); break;
            }
            __syncthreads();
            be = 0.0;
            for (int c = 0; c < rc; ++c) {
                const double rm = rmax[c], xm = xmax[c];
                const double e = (an > 0.0 && xm > 0.0) ? rm / (an * xm) : (rm > 0.0 ? INFINITY : 0.0);
                if (!(e <= be)) be = e;
            }
            if (be <= a.tol || it >= a.max_iter) break;
            ++it;
            for (int e = tid; e < n * rc; e += bt::THREADS) {
                const int i = e % n, c = e / n;
                y[(size_t)c * nmax + i] = (TL)tmp[(size_t)c * nmax + i];
            }
            __syncthreads();
            bt_solve<TL>(n, rc, nmax, L, ldl, a.Dd[sys], a.Ds[sys], a.perm[sys], y, tmp);
            for (int e = tid; e < n * rc; e += bt::THREADS) {
                const int i = e % n, c = e / n;
                x[(size_t)c * nmax + i] += (double)y[(size_t)c * nmax + i];
            }
            __syncthreads();
        }
        for (int e = tid; e < n * rc; e += bt::THREADS) {
            const int i = e % n, c = e / n;
            X[(size_t)i + (size_t)(c0 + c) * ldx] = x[(size_t)c * nmax + i];
        }
        if (!(be <= worst)) worst = be;
        if (it > most) most = it;
        __syncthreads();
    }
    if (tid == 0) {
        if (a.berr) a.berr[sys] = A64 ? worst : 0.0;
        if (a.iters) a.iters[sys] = most;
    }
}

template <typename TL>
__global__ void __launch_bounds__(bt::THREADS, 1) batched_refine_kernel(BtRefineArgs<TL> a) {
    extern __shared__ __align__(16) unsigned char br_raw[];
    __shared__ double s_an;
    __shared__ int s_idx;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(a.ticket, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= a.batch) return;
        bt_refine_one<TL>(a, a.order[idx], br_raw, &s_an);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// order: systems by decreasing n (counting sort in one CTA), and the launchers
// ---------------------------------------------------------------------------------------------
__global__ void batched_order_kernel(int batch, int nmax, const int *n, int *order) {
    extern __shared__ int cnt[];   // nmax + 1 counters
    for (int v = threadIdx.x; v <= nmax; v += blockDim.x) cnt[v] = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < batch; s += blockDim.x) atomicAdd(&cnt[nmax - min(max(n[s], 0), nmax)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int v = 0; v <= nmax; ++v) { const int c = cnt[v]; cnt[v] = run; run += c; }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < batch; s += blockDim.x)
        order[atomicAdd(&cnt[nmax - min(max(n[s], 0), nmax)], 1)] = s;
}

static int bt_grid(const void *fn, size_t smem, int batch) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, bt::THREADS, smem);
    const long long g = (long long)sms * (per > 0 ? per : 1);
    return (int)(g < batch ? g : batch);
}

cudaError_t launch_batched_order(int batch, int nmax, const int *n, int *order, cudaStream_t s) {
    batched_order_kernel<<<1, 1024, (size_t)(nmax + 1) * sizeof(int), s>>>(batch, nmax, n, order);
    count_launches(1);
    return cudaGetLastError();
}

size_t batched_max_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v > 1024 ? (size_t)v - 1024 : 0;   // room for the kernels' static shared memory
}

template <typename T>
cudaError_t launch_batched_factor(int batch, int d, int b, int nmax, const int *n, const double *const *A64,
                                  const int *lda64, T *const *A, const int *lda, double *const *Dd, double *const *Ds,
                                  int *const *perm, const T *om, double alpha, int *info, const int *order,
                                  int *ticket, cudaStream_t s) {
    BtFactorArgs<T> a{batch, d, b, nmax, n, A64, lda64, A, lda, Dd, Ds, perm, om, alpha, info, order, ticket};
    const size_t smem = batched_factor_smem<T>(d, b, nmax);
    cudaError_t e = cudaFuncSetAttribute(batched_factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ticket, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    batched_factor_kernel<T><<<bt_grid((const void *)batched_factor_kernel<T>, smem, batch), bt::THREADS, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <typename TL>
cudaError_t launch_batched_refine(int batch, int nrhs, int nmax, int max_iter, double tol, const int *n,
                                  const TL *const *LA, const int *ldla, const double *const *Dd,
                                  const double *const *Ds, const int *const *perm, const double *const *A64,
                                  const int *lda64, const double *const *Bv, const int *ldb, double *const *X,
                                  const int *ldx, double *berr, int *iters, const int *order, int *ticket,
                                  cudaStream_t s) {
    BtRefineArgs<TL> a{batch, nrhs, nmax, max_iter, tol, n, LA, ldla, Dd, Ds, perm, A64, lda64, Bv, ldb, X, ldx,
                       berr, iters, order, ticket};
    const size_t smem = batched_refine_smem<TL>(nrhs, nmax);
    cudaError_t e = cudaFuncSetAttribute(batched_refine_kernel<TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ticket, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    batched_refine_kernel<TL><<<bt_grid((const void *)batched_refine_kernel<TL>, smem, batch), bt::THREADS, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

#define BT_INST(T)                                                                                                   \
    template size_t batched_factor_smem<T>(int, int, int);                                                           \
    template size_t batched_refine_smem<T>(int, int);                                                                \
    template cudaError_t launch_batched_factor<T>(int, int, int, int, const int *, const double *const *, const int *, \
                                                  T *const *, const int *, double *const *, double *const *,          \
                                                  int *const *, const T *, double, int *, const int *, int *,         \
                                                  cudaStream_t);                                                     \
    template cudaError_t launch_batched_refine<T>(int, int, int, int, double, const int *, const T *const *,          \
                                                  const int *, const double *const *, const double *const *,          \
                                                  const int *const *, const double *const *, const int *,             \
                                                  const double *const *, const int *, double *const *, const int *,   \
                                                  double *, int *, const int *, int *, cudaStream_t);
BT_INST(float)
BT_INST(double)
#undef BT_INST

}  // namespace rcpk
