// batched.cu -- many independent small systems (n <= a few hundred): RCP factorization and
// FP64 iterative refinement, one persistent kernel per phase.
//
// Each CTA takes systems from an atomic ticket; the order puts the largest systems first
// (longest-processing-time-first scheduling), so the tail of the launch is made of small
// systems.  One CTA runs Algorithm 1 (q = 1) on one system, so every synchronization of the
// method is a CTA barrier, and the per-system state (sketch, panel) lives in shared memory.
// The factor's CTAs have 512, 256 or 128 threads: a pivot step waits on a dependent load of A
// and on CTA barriers, so two or more smaller CTAs per SM overlap several systems' waits (a
// thread then owns several positions of a step and issues all their loads of A at once).  A
// split schedule runs the systems above an order in one launch of 512-thread CTAs and the rest
// in a second launch of 256-thread CTAs sized for the smaller order.  The shared state of one
// system:
//
//   Bs   nmax x dp     the sketch B = Omega A, one column per row ([j][r], dp = d rounded up to
//                      a multiple of 4, padding zero), updated after every pivot
//   W    (b+1) x nmax  Schur-complement columns of the current panel ([t][j])
//   Lp   (b+1) x nmax  the panel's multipliers ([t][j])
//   c1, c2            the Schur columns k and r of the current step
//   stg  4 x dp        sketch columns staged for the interchanges of the step
//
// A itself (lower triangle, column-major) stays in global memory.  A pivot step is two or
// three barrier phases:
//   A  interchange k <-> P in the trailing part of A (global), Schur column k, argmax |c1|
//   R  (SBKP cases 2 and 3 only) Schur column r, the case decision, the 2x2 inverse (FP64)
//   B  multipliers, panel columns, rank-s sketch update and column norms, argmax of the norms;
//      the second interchange of cases 2 and 3 is applied to the trailing part of A here
// The interchanges of the sketch, W and Lp are relabellings resolved in phase B (the columns
// they move are staged first).  Row interchanges of the columns already factored are not
// applied during the factorization: the permutation at the end of every panel is recorded,
// and one pass at the end permutes the rows of every panel's L columns (the deferred row
// interchanges of LAPACK's blocked factorizations).  The panel's trailing update
// A22 -= W Lp^T runs at the end of every panel.  The omega matrix is drawn once per call
// (d x nmax); system i uses its first n_i columns, which are the columns a d x n_i draw with
// the same seed gives.
#include <cfloat>
#include <climits>

#include "kernels.h"

namespace rcpk {

namespace bt {
constexpr int THREADS = 512;
constexpr int WARPS = THREADS / 32;
constexpr int TILE = 32;          // sketch tiles
constexpr int MR = 128 / WARPS;   // sketch rows per thread: d <= WARPS * MR = 128
constexpr unsigned FULLM = 0xffffffffu;
}  // namespace bt

// ---------------------------------------------------------------------------------------------
// block-wide argmax (value descending, index ascending), one barrier per call
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
struct BtShared {
    BtCand<T> red[2][bt::WARPS];      // FP64: per-warp candidates, two buffers used alternately
    unsigned long long key[3];        // FP32: packed keys, three slots used in rotation
    T sc2[4];                         // 2x2 inverse entries of the current step
    int kase;                         // SBKP case decided in phase R
    int s_idx;
};

// FP64: warp shuffles, then every thread reduces the NW warp candidates.
template <int NW>
__device__ __forceinline__ BtCand<double> bt_argmax(BtCand<double> c, BtShared<double> &sh, int &cnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, buf = cnt & 1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double v = __shfl_xor_sync(bt::FULLM, c.v, off);
        const int j = __shfl_xor_sync(bt::FULLM, c.j, off);
        if (bt_better(v, j, c.v, c.j)) { c.v = v; c.j = j; }
    }
    if (lane == 0) sh.red[buf][warp] = c;
    __syncthreads();
    BtCand<double> r = sh.red[buf][0];
#pragma unroll
    for (int w2 = 1; w2 < NW; ++w2) {
        const BtCand<double> x = sh.red[buf][w2];
        if (bt_better(x.v, x.j, r.v, r.j)) r = x;
    }
    ++cnt;
    return r;
}

// FP32, values >= 0: the key (value bits << 32) | ~j orders like (value desc, index asc); a
// warp takes its maximum with two redux.sync, the block with one shared 64-bit atomicMax.
// Slot cnt % 3 serves this call; the slot of the next call, last read two barriers ago, is
// cleared here.  A NaN value wins (its bits exceed those of +Inf), so the caller sees it.
template <int NW>
__device__ __forceinline__ BtCand<float> bt_argmax(BtCand<float> c, BtShared<float> &sh, int &cnt) {
    const bool has = c.j != INT_MAX;
    const unsigned hi = has ? __float_as_uint(c.v) : 0u, lo = has ? ~(unsigned)c.j : 0u;
    const unsigned m = __reduce_max_sync(bt::FULLM, hi);
    const unsigned l = __reduce_max_sync(bt::FULLM, hi == m ? lo : 0u);
    const int slot = cnt % 3;
    if (threadIdx.x == 0) sh.key[(cnt + 1) % 3] = 0ull;
    if ((threadIdx.x & 31) == 0) atomicMax(&sh.key[slot], ((unsigned long long)m << 32) | l);
    __syncthreads();
    const unsigned long long kk = sh.key[slot];
    ++cnt;
    BtCand<float> r;
    r.v = __uint_as_float((unsigned)(kk >> 32));
    r.j = (unsigned)kk == 0u ? INT_MAX : (int)(~(unsigned)kk);
    return r;
}

template <typename T>
__device__ __forceinline__ T bt_abs(T x) { return x < T(0) ? -x : x; }

template <typename T>
__device__ __forceinline__ T a_sym(const T *A, int lda, int i, int j) {
    return i >= j ? A[(size_t)i + (size_t)j * lda] : A[(size_t)j + (size_t)i * lda];
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
    int *pscr;                  // per CTA: panel bounds and the permutation after every panel
    const int *first, *last;    // device: the range of order[] this launch takes (NULL: 0, batch)
};

// panels of one system: widths b or b + 1, so at most nmax / b + 1 of them
__host__ __device__ inline int bt_max_panels(int b, int nmax) { return nmax / b + 2; }

size_t batched_factor_scratch_ints(int b, int nmax) {
    return (size_t)bt_max_panels(b, nmax) * (nmax + 1) + 16;
}

// row stride of the shared arrays: nmax rounded up to a multiple of 4 (16-byte rows for FP32)
__host__ __device__ inline int bt_stride(int nmax) { return (nmax + 3) & ~3; }

// shared-memory elements of type T for one system of order <= nmax: Bs, W and Lp (the sketch
// tiles alias W and Lp), c1, c2, the staged sketch columns and the permutation (ints)
__host__ __device__ inline size_t bt_factor_elems(int d, int b, int nmax) {
    const size_t ns = bt_stride(nmax), dp = bt_stride(d);
    const size_t panel = 2 * (size_t)(b + 1) * ns;
    const size_t sk = ((size_t)(bt::TILE + d) * (bt::TILE + 1) + 3) & ~(size_t)3;
    return dp * ns + (panel > sk ? panel : sk) + 2 * ns + 4 * dp + ns;
}

template <typename T>
size_t batched_factor_smem(int d, int b, int nmax) {
    return bt_factor_elems(d, b, nmax) * sizeof(T);
}

// DR > 0: thread j keeps the sketch column of position j in registers (n <= NT, dp <= DR,
// FP32 only); DR == 0: the sketch stays in shared memory.
template <typename T, int DR, int NT>
__device__ void bt_factor_one(const BtFactorArgs<T> &a, int sys, T *sm, BtShared<T> &sh, int &cnt) {
    static_assert(DR == 0 || (sizeof(T) == 4 && DR % 4 == 0), "register sketch: FP32, whole float4s");
    constexpr int DR4 = DR > 0 ? DR / 4 : 1;
    constexpr int RU = NT >= 512 ? 1 : 512 / NT;   // positions per thread whose loads go out together
    constexpr int NW = NT / 32, MR = 128 / NW;     // warps; sketch rows per thread (d <= NW * MR = 128)
    float4 b4[DR4];   // the register sketch column (DR > 0)
    const int n = a.n[sys], d = a.d, nmax = bt_stride(a.nmax), tid = threadIdx.x;
    const int lda = a.lda[sys];
    T *A = a.A[sys];
    double *Dd = a.Dd[sys], *Ds = a.Ds[sys];
    int *perm_out = a.perm[sys];
    if (n <= 0) {
        if (tid == 0) a.info[sys] = 0;
        return;
    }
    // nmax below is the padded row stride of the shared arrays
    const int dp = bt_stride(d);
    const size_t panel = 2 * (size_t)(a.b + 1) * nmax;
    const size_t skel = ((size_t)(bt::TILE + d) * (bt::TILE + 1) + 3) & ~(size_t)3;   // 16-byte multiple
    T *Bs = sm;                                        // [nmax][dp]
    T *W = Bs + (size_t)dp * nmax;                     // [b+1][nmax]
    T *Lp = W + (size_t)(a.b + 1) * nmax;              // [b+1][nmax]
    T *c1 = W + (panel > skel ? panel : skel);
    T *c2 = c1 + nmax;
    T *stg = c2 + nmax;                                // [4][dp]: old sketch columns k, k+1, P, r
    int *perm = reinterpret_cast<int *>(stg + 4 * dp); // [nmax]: the permutation
    const int npmax = bt_max_panels(a.b, a.nmax);
    int *pbound = a.pscr + (size_t)blockIdx.x * (npmax * (size_t)(a.nmax + 1) + 16);
    int *psnap = pbound + npmax + 1;                   // [panel][a.nmax]

    // ---- optional FP64 source: copy the lower triangle into the factor array ----
    if (a.A64) {
        const double *S = a.A64[sys];
        const int lds = a.lda64[sys];
        for (int e = tid; e < n * n; e += NT) {
            const int i = e % n, j = e / n;
            if (i >= j) A[(size_t)i + (size_t)j * lda] = (T)S[(size_t)i + (size_t)j * lds];
        }
    }
    for (int x = tid; x < n; x += NT) perm[x] = x;
    __syncthreads();

    // ---- B = Omega(:, 0:n) A by 32 x 32 tiles of A (the sketch region aliases the panels) ----
    {
        T *As = W;                                     // [32][33]: As[i][j] = A_sym(i0 + i, j0 + j)
        T *Os = W + bt::TILE * (bt::TILE + 1);         // [d][33]:  Os[r][i] = Omega(r, i0 + i)
        const int jj = tid & 31, r0 = tid >> 5;
        for (int j0 = 0; j0 < n; j0 += bt::TILE) {
            T acc[MR];
#pragma unroll
            for (int m = 0; m < MR; ++m) acc[m] = T(0);
            for (int i0 = 0; i0 < n; i0 += bt::TILE) {
                for (int e = tid; e < bt::TILE * bt::TILE; e += NT) {
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
                for (int e = tid; e < d * bt::TILE; e += NT) {
                    const int r = e % d, i = e / d;
                    Os[r * (bt::TILE + 1) + i] = (i0 + i < n) ? a.om[(size_t)r + (size_t)(i0 + i) * d] : T(0);
                }
                __syncthreads();
#pragma unroll 4
                for (int i = 0; i < bt::TILE; ++i) {
                    const T av = As[i * (bt::TILE + 1) + jj];
#pragma unroll
                    for (int m = 0; m < MR; ++m) {
                        const int r = r0 + NW * m;
                        if (r < d) acc[m] += Os[r * (bt::TILE + 1) + i] * av;
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int r = r0 + NW * m;
                if (r < dp && j0 + jj < n) Bs[(size_t)(j0 + jj) * dp + r] = r < d ? acc[m] : T(0);
            }
        }
    }
    __syncthreads();

    // ---- first pivot candidate: max column norm of B ----
    BtCand<T> cand{T(-1), INT_MAX};
    if constexpr (DR > 0) {
        if (tid < n) {
            const float4 *c4 = reinterpret_cast<const float4 *>(Bs + (size_t)tid * dp);
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int q = 0; q < DR4; ++q) {
                b4[q] = 4 * q < dp ? c4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                s0 += b4[q].x * b4[q].x + b4[q].z * b4[q].z;
                s1 += b4[q].y * b4[q].y + b4[q].w * b4[q].w;
            }
            cand = BtCand<T>{(T)(s0 + s1), tid};
        }
    } else {
        for (int j = tid; j < n; j += NT) {
            T s = T(0);
            for (int r = 0; r < d; ++r) { const T v = Bs[(size_t)j * dp + r]; s += v * v; }
            if (bt_better(s, j, cand.v, cand.j)) cand = BtCand<T>{s, j};
        }
    }
    cand = bt_argmax<NW>(cand, sh, cnt);

    int info = 0, k = 0, np = 0;
    bool bad = false;
    const T alpha = (T)a.alpha;
    while (k < n && !bad) {
        const int k0 = k;
        int i = 0;
        while (i < a.b && k < n) {
            const int P = cand.j;
            if (P < k || P >= n || !isfinite(cand.v)) { bad = true; break; }
            // ---- phase A: k <-> P in the trailing part of A; Schur column k in the new labels
            //      (W, Lp and Bs are still in the old labels: position x came from sigma(x)) ----
            BtCand<T> lc{T(-1), INT_MAX};
            // RU positions per thread at a time: all their loads of A are issued before any store
            // (no two positions touch the same entry), so a thread waits for one round trip
            for (int xb = k + tid; xb < n; xb += RU * NT) {
                T av[RU], ak[RU];
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int x = xb + u * NT;
                    if (x >= n) continue;
                    if (x == k) {
                        av[u] = A[(size_t)P + (size_t)P * lda];
                        if (P != k) ak[u] = A[(size_t)k + (size_t)k * lda];
                    } else if (x == P) {
                        av[u] = A[(size_t)P + (size_t)k * lda];
                    } else {
                        av[u] = x > P ? A[(size_t)x + (size_t)P * lda] : A[(size_t)P + (size_t)x * lda];
                        if (P != k) ak[u] = A[(size_t)x + (size_t)k * lda];
                    }
                }
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int x = xb + u * NT;
                    if (x >= n) continue;
                    if (P != k && x != P) {
                        if (x == k) {
                            A[(size_t)P + (size_t)P * lda] = ak[u];
                            A[(size_t)k + (size_t)k * lda] = av[u];
                        } else {
                            T *up = x > P ? A + (size_t)x + (size_t)P * lda : A + (size_t)P + (size_t)x * lda;
                            *up = ak[u];
                            A[(size_t)x + (size_t)k * lda] = av[u];
                        }
                    }
                    // the panel's correction does not wait for the load of A
                    const int sx = x == k ? P : (x == P ? k : x);
                    T cs = T(0);
#pragma unroll 8
                    for (int t = 0; t < i; ++t) cs += W[(size_t)t * nmax + sx] * Lp[(size_t)t * nmax + P];
                    const T v = av[u] - cs;
                    c1[x] = v;
                    if (x > k && bt_better(bt_abs(v), x, lc.v, lc.j)) lc = BtCand<T>{bt_abs(v), x};
                }
            }
            if constexpr (DR > 0) {
                // the owners of positions k and P stage their columns
                if (tid == k || tid == P) {
                    float4 *o0 = reinterpret_cast<float4 *>(stg), *o2 = reinterpret_cast<float4 *>(stg + 2 * dp);
#pragma unroll
                    for (int q = 0; q < DR4; ++q) {
                        if (4 * q < dp) {
                            if (tid == k) o0[q] = b4[q];
                            if (tid == P) o2[q] = b4[q];
                        }
                    }
                }
            } else {
                for (int e = tid; e < 2 * dp; e += NT) {
                    const int r = e < dp ? e : e - dp;
                    stg[e < dp ? r : 2 * dp + r] = Bs[(size_t)(e < dp ? k : P) * dp + r];
                }
            }
            lc = bt_argmax<NW>(lc, sh, cnt);
            // ---- SBKP decision (every thread, in the factor's type) ----
            const int R = lc.j < n ? lc.j : -1;     // new label
            const T lam = R >= 0 ? lc.v : T(0);
            const T akk = c1[k];
            if (!isfinite(lam) || !isfinite(akk)) { bad = true; break; }
            int kase;
            if (R < 0 || lam == T(0)) kase = 0;
            else if (bt_abs(akk) >= alpha * lam) kase = 1;
            else kase = 4;
            const int sR = R < 0 ? -1 : (R == P ? k : R);   // old label of R
            if (kase == 4) {
                // ---- phase R: Schur column R (new labels), decision, 2x2 inverse, staging ----
                for (int xb = k + tid; xb < n; xb += RU * NT) {
                T avr[RU];
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int x = xb + u * NT;
                    if (x < n) avr[u] = a_sym(A, lda, x, R);
                }
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int x = xb + u * NT;
                    if (x >= n) continue;
                    const int sx = x == k ? P : (x == P ? k : x);
                    T cs = T(0);
#pragma unroll 8
                    for (int t = 0; t < i; ++t) cs += W[(size_t)t * nmax + sx] * Lp[(size_t)t * nmax + sR];
                    const T av = avr[u] - cs;
                    c2[x] = av;
                    if (x == R) {
                        int kk;
                        if (!isfinite(av)) kk = -1;
                        else if (bt_abs(av) >= alpha * lam) kk = 2;
                        else kk = 3;
                        if (kk == 3) {
                            // D = [[a11, a21], [a21, a22]] with |det| >= (1 - alpha^2) lam^2:
                            // one FP64 division gives D^{-1} = [[a22, -a21], [-a21, a11]] / det
                            const double a11 = (double)c1[k], a21 = (double)c1[R], a22 = (double)av;
                            const double rdet = 1.0 / fma(a11, a22, -a21 * a21);
                            sh.sc2[0] = (T)(a22 * rdet);
                            sh.sc2[1] = (T)(-a21 * rdet);
                            sh.sc2[2] = (T)(a11 * rdet);
                            Dd[k] = a11; Ds[k] = a21; Dd[k + 1] = a22; Ds[k + 1] = 0.0;
                        } else if (kk == 2) {
                            Dd[k] = (double)av;
                            Ds[k] = 0.0;
                        }
                        sh.kase = kk;
                    }
                }
                }
                if constexpr (DR > 0) {
                    if (tid == k + 1 || tid == sR) {
                        float4 *o1 = reinterpret_cast<float4 *>(stg + dp), *o3 = reinterpret_cast<float4 *>(stg + 3 * dp);
#pragma unroll
                        for (int q = 0; q < DR4; ++q) {
                            if (4 * q < dp) {
                                if (tid == k + 1) o1[q] = b4[q];
                                if (tid == sR) o3[q] = b4[q];
                            }
                        }
                    }
                } else {
                    for (int e = tid; e < 2 * dp; e += NT) {
                        const int r = e < dp ? e : e - dp;
                        stg[e < dp ? dp + r : 3 * dp + r] = Bs[(size_t)(e < dp ? k + 1 : sR) * dp + r];
                    }
                }
                __syncthreads();
                kase = sh.kase;
                if (kase < 0) { bad = true; break; }
            }
            // ---- phase B ----
            const int s = kase == 3 ? 2 : 1;
            const int tgt = kase == 2 ? k : (kase == 3 ? k + 1 : -1);
            const int Rm = (kase >= 2 && R != tgt) ? R : -1;       // new label moved by the 2nd interchange
            const T *cp = kase == 2 ? c2 : c1;
            const T *pbA = stg + (kase == 2 ? 3 * dp : 2 * dp), *pbB = stg + 3 * dp;
            T finv = T(0), f11 = T(0), f21 = T(0), f22 = T(0);
            if (s == 1) {
                const T dp = cp[kase == 2 ? R : k];
                if (kase < 2 && tid == 0) {
                    Dd[k] = (double)dp;
                    Ds[k] = 0.0;
                }
                if (dp == T(0) && info == 0) info = k + 1;
                finv = dp != T(0) ? T(1) / dp : T(0);
            } else {
                f11 = sh.sc2[0]; f21 = sh.sc2[1]; f22 = sh.sc2[2];
            }
            // the second interchange, tgt <-> R, in the trailing part of A: position R gets the
            // row and column of tgt (tgt becomes a pivot position, its own entries are dead); the
            // loads are issued here and the stores after the loop below
            T mv = T(0);
            T *mdst = nullptr;
            if (Rm >= 0) {
                const int x = k + s + tid;     // the first element of each thread; any others below
                if (x < n) {
                    if (x == Rm) { mv = A[(size_t)tgt + (size_t)tgt * lda]; mdst = A + (size_t)Rm + (size_t)Rm * lda; }
                    else {
                        mv = A[(size_t)x + (size_t)tgt * lda];
                        mdst = x > Rm ? A + (size_t)x + (size_t)Rm * lda : A + (size_t)Rm + (size_t)x * lda;
                    }
                }
            }
            BtCand<T> nc{T(-1), INT_MAX};
            if constexpr (DR > 0) {
                const int j = tid;
                if (j >= k + s && j < n) {
                    const int u = j == Rm ? tgt : j;                   // label after the first interchange
                    const int o = u == k ? P : (u == P ? k : u);         // label before the step
                    float l1, l2 = 0.f;
                    if (s == 1) {
                        const T cj = cp[u];
                        l1 = cj * finv;
                        W[(size_t)i * nmax + j] = cj;
                        Lp[(size_t)i * nmax + j] = l1;
                    } else {
                        const T x1 = c1[u], x2 = c2[u];
                        l1 = f11 * x1 + f21 * x2;
                        l2 = f21 * x1 + f22 * x2;
                        W[(size_t)i * nmax + j] = x1;
                        W[(size_t)(i + 1) * nmax + j] = x2;
                        Lp[(size_t)i * nmax + j] = l1;
                        Lp[(size_t)(i + 1) * nmax + j] = l2;
                    }
                    if (o != j) {
                        // this position receives a column moved by the interchanges (staged)
                        const float4 *src4 = reinterpret_cast<const float4 *>(
                            stg + (o == k ? 0 : (o == k + 1 ? dp : (o == P ? 2 * dp : 3 * dp))));
#pragma unroll
                        for (int q = 0; q < DR4; ++q)
                            if (4 * q < dp) b4[q] = src4[q];
                    }
                    const float4 *a4 = reinterpret_cast<const float4 *>(pbA);
                    const float4 *q4 = reinterpret_cast<const float4 *>(pbB);
                    float n0 = 0.f, n1 = 0.f;
#pragma unroll
                    for (int q = 0; q < DR4; ++q) {
                        if (4 * q < dp) {
                            const float4 pa = a4[q];
                            float4 v = b4[q];
                            v.x -= pa.x * l1; v.y -= pa.y * l1; v.z -= pa.z * l1; v.w -= pa.w * l1;
                            if (s == 2) {
                                const float4 pq = q4[q];
                                v.x -= pq.x * l2; v.y -= pq.y * l2; v.z -= pq.z * l2; v.w -= pq.w * l2;
                            }
                            b4[q] = v;
                            n0 += v.x * v.x + v.z * v.z;
                            n1 += v.y * v.y + v.w * v.w;
                        }
                    }
                    nc = BtCand<T>{(T)(n0 + n1), j};
                }
            } else {
                for (int j = k + s + tid; j < n; j += NT) {
                    const int u = j == Rm ? tgt : j;                   // label after the first interchange
                    const int o = u == k ? P : (u == P ? k : u);         // label before the step
                    const T *src = o == j ? Bs + (size_t)j * dp
                                          : stg + (o == k ? 0 : (o == k + 1 ? dp : (o == P ? 2 * dp : 3 * dp)));
                    T *dst = Bs + (size_t)j * dp;
                    T l1, l2 = T(0);
                    if (s == 1) {
                        const T cj = cp[u];
                        l1 = cj * finv;
                        W[(size_t)i * nmax + j] = cj;
                        Lp[(size_t)i * nmax + j] = l1;
                    } else {
                        const T x1 = c1[u], x2 = c2[u];
                        l1 = f11 * x1 + f21 * x2;
                        l2 = f21 * x1 + f22 * x2;
                        W[(size_t)i * nmax + j] = x1;
                        W[(size_t)(i + 1) * nmax + j] = x2;
                        Lp[(size_t)i * nmax + j] = l1;
                        Lp[(size_t)(i + 1) * nmax + j] = l2;
                    }
                    T nrm0 = T(0), nrm1 = T(0);
                    if constexpr (sizeof(T) == 4) {
                        // 16-byte rows: the column, the pivot columns and the update move as float4
                        const float4 *s4 = reinterpret_cast<const float4 *>(src);
                        const float4 *a4 = reinterpret_cast<const float4 *>(pbA);
                        const float4 *b4 = reinterpret_cast<const float4 *>(pbB);
                        float4 *d4 = reinterpret_cast<float4 *>(dst);
                        if (s == 1) {
    #pragma unroll 2
                            for (int r4 = 0; r4 < dp / 4; ++r4) {
                                float4 v = s4[r4];
                                const float4 pa = a4[r4];
                                v.x -= pa.x * l1; v.y -= pa.y * l1; v.z -= pa.z * l1; v.w -= pa.w * l1;
                                d4[r4] = v;
                                nrm0 += v.x * v.x + v.z * v.z;
                                nrm1 += v.y * v.y + v.w * v.w;
                            }
                        } else {
    #pragma unroll 2
                            for (int r4 = 0; r4 < dp / 4; ++r4) {
                                float4 v = s4[r4];
                                const float4 pa = a4[r4], pq = b4[r4];
                                v.x -= pa.x * l1 + pq.x * l2; v.y -= pa.y * l1 + pq.y * l2;
                                v.z -= pa.z * l1 + pq.z * l2; v.w -= pa.w * l1 + pq.w * l2;
                                d4[r4] = v;
                                nrm0 += v.x * v.x + v.z * v.z;
                                nrm1 += v.y * v.y + v.w * v.w;
                            }
                        }
                    } else {
                        for (int r = 0; r < d; ++r) {
                            T w = src[r] - pbA[r] * l1;
                            if (s == 2) w -= pbB[r] * l2;
                            dst[r] = w;
                            if (r & 1) nrm1 += w * w; else nrm0 += w * w;
                        }
                    }
                    const T nrm = nrm0 + nrm1;
                    if (bt_better(nrm, j, nc.v, nc.j)) nc = BtCand<T>{nrm, j};
                }
            }
            // the interchanges of the panel rows: new row q of W and Lp is old row sigma(tau(q))
            for (int e = tid; e < 2 * i; e += NT) {
                T *rowp = (e < i ? W : Lp) + (size_t)(e < i ? e : e - i) * nmax;
                const int q4[4] = {k, P, k + 1 < n ? k + 1 : k, Rm >= 0 ? Rm : k};
                T v4[4];
#pragma unroll
                for (int z = 0; z < 4; ++z) {
                    const int u = q4[z] == Rm ? tgt : (q4[z] == tgt ? Rm : q4[z]);
                    const int uu = Rm < 0 ? q4[z] : u;
                    v4[z] = rowp[uu == k ? P : (uu == P ? k : uu)];
                }
#pragma unroll
                for (int z = 0; z < 4; ++z) rowp[q4[z]] = v4[z];
            }
            if (tid == 0) {
                if (P != k) { const int t = perm[k]; perm[k] = perm[P]; perm[P] = t; }
                if (Rm >= 0) { const int t = perm[tgt]; perm[tgt] = perm[Rm]; perm[Rm] = t; }
            }
            if (s == 2 && tid == 0) Lp[(size_t)i * nmax + k + 1] = T(0);   // L(k+1, k) of a 2x2 block
            if (mdst) *mdst = mv;
            if (Rm >= 0) {
                for (int x = k + s + tid + NT; x < n; x += NT) {
                    if (x == Rm) A[(size_t)Rm + (size_t)Rm * lda] = A[(size_t)tgt + (size_t)tgt * lda];
                    else if (x > Rm) A[(size_t)x + (size_t)Rm * lda] = A[(size_t)x + (size_t)tgt * lda];
                    else A[(size_t)Rm + (size_t)x * lda] = A[(size_t)x + (size_t)tgt * lda];
                }
            }
            cand = bt_argmax<NW>(nc, sh, cnt);
            k += s;
            i += s;
        }
        if (bad) break;
        // ---- end of the panel: multipliers into A, the permutation so far, A22 -= W Lp^T ----
        for (int e = tid; e < i * (n - k0); e += NT) {
            const int t = e / (n - k0), p = k0 + e % (n - k0);
            if (p > k0 + t) A[(size_t)p + (size_t)(k0 + t) * lda] = Lp[(size_t)t * nmax + p];
        }
        if (k < n) {
            for (int x = tid; x < n; x += NT) psnap[(size_t)np * a.nmax + x] = perm[x];
            if (tid == 0) pbound[np] = k;
            ++np;
        }
        if (n - k > 0) {
            // 4 x 4 tiles of the lower triangle of A(k:n, k:n) from an aligned start kA; tile
            // (I, J), I >= J, enumerated so that consecutive threads take consecutive row tiles
            // of one column tile (coalesced columns of A)
            const int kA = k & ~3, nt = (n - kA + 3) >> 2, ntri = nt * (nt + 1) / 2;
            for (int tt = tid; tt < ntri; tt += NT) {
                int ra = (int)((sqrtf(8.f * (float)tt + 1.f) - 1.f) * 0.5f);
                while (ra * (ra + 1) / 2 > tt) --ra;
                while ((ra + 1) * (ra + 2) / 2 <= tt) ++ra;
                const int rb = tt - ra * (ra + 1) / 2;
                const int J = nt - 1 - ra, I = nt - 1 - rb;
                const int p0 = kA + 4 * I, q0 = kA + 4 * J;
                T acc[4][4];
#pragma unroll
                for (int y = 0; y < 4; ++y)
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const int p = p0 + x, q = q0 + y;
                        acc[x][y] = (p < n && q >= k && p >= q) ? A[(size_t)p + (size_t)q * lda] : T(0);
                    }
                for (int t = 0; t < i; ++t) {
                    T wv[4], lv[4];
                    if constexpr (sizeof(T) == 4) {
                        const float4 w4 = *reinterpret_cast<const float4 *>(W + (size_t)t * nmax + p0);
                        const float4 l4 = *reinterpret_cast<const float4 *>(Lp + (size_t)t * nmax + q0);
                        wv[0] = w4.x; wv[1] = w4.y; wv[2] = w4.z; wv[3] = w4.w;
                        lv[0] = l4.x; lv[1] = l4.y; lv[2] = l4.z; lv[3] = l4.w;
                    } else {
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            wv[x] = W[(size_t)t * nmax + p0 + x];
                            lv[x] = Lp[(size_t)t * nmax + q0 + x];
                        }
                    }
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] -= wv[x] * lv[y];
                }
#pragma unroll
                for (int y = 0; y < 4; ++y)
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const int p = p0 + x, q = q0 + y;
                        if (p < n && q >= k && p >= q) A[(size_t)p + (size_t)q * lda] = acc[x][y];
                    }
            }
        }
        __syncthreads();
    }
    if (bad) {
        for (int x = tid; x < n; x += NT) perm_out[x] = perm[x];
        if (tid == 0) a.info[sys] = BT_INFO_NONFINITE;
        __syncthreads();
        return;
    }
    // ---- deferred row interchanges: rows q >= end of panel J of that panel's L columns hold
    //      the row that sat at position inv_J[perm[q]] when the panel ended ----
    {
        int *pf = reinterpret_cast<int *>(W);          // final permutation
        int *inv = pf + nmax;                          // inverse of the panel's permutation
        for (int x = tid; x < n; x += NT) pf[x] = perm[x];
        int c0 = 0;
        for (int J = 0; J < np; ++J) {
            const int kend = pbound[J];
            __syncthreads();
            for (int x = tid; x < n; x += NT) inv[psnap[(size_t)J * a.nmax + x]] = x;
            for (int cb = c0; cb < kend; cb += d) {
                const int cw = min(d, kend - cb), rows = n - kend;
                __syncthreads();
                for (int e = tid; e < cw * rows; e += NT) {
                    const int q = kend + e % rows, c = cb + e / rows;
                    Bs[(size_t)(e / rows) * nmax + q] = A[(size_t)q + (size_t)c * lda];
                }
                __syncthreads();
                for (int e = tid; e < cw * rows; e += NT) {
                    const int q = kend + e % rows, c = cb + e / rows;
                    A[(size_t)q + (size_t)c * lda] = Bs[(size_t)(e / rows) * nmax + inv[pf[q]]];
                }
            }
            c0 = kend;
        }
    }
    for (int x = tid; x < n; x += NT) {
        A[(size_t)x + (size_t)x * lda] = (T)Dd[x];
        perm_out[x] = perm[x];
    }
    if (tid == 0) a.info[sys] = info;
    __syncthreads();
}

// NT threads per CTA: 512 (one CTA per SM), 256 or 128 (two, or up to four, per SM where the
// shared memory allows).
// The CTAs take the systems order[first .. last) (first and last read from device memory when
// given, else 0 and batch).
template <typename T, int DR, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) batched_factor_kernel(BtFactorArgs<T> a) {
    static_assert(NT == 128 || NT == 256 || NT == 512, "CTA size");
    extern __shared__ __align__(16) unsigned char bt_raw[];
    __shared__ BtShared<T> sh;
    int cnt = 0;
    if (threadIdx.x == 0) { sh.key[0] = sh.key[1] = sh.key[2] = 0ull; }
    const int first = a.first ? *a.first : 0, last = a.last ? *a.last : a.batch;
    for (;;) {
        if (threadIdx.x == 0) sh.s_idx = first + atomicAdd(a.ticket, 1);
        __syncthreads();
        const int idx = sh.s_idx;
        __syncthreads();
        if (idx >= last) return;
        bt_factor_one<T, DR, NT>(a, a.order[idx], reinterpret_cast<T *>(bt_raw), sh, cnt);
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
constexpr int BT_YS = 20;       // row stride of y: 16 right-hand sides + 4 (conflict-free 16-byte rows)
constexpr int BT_LS = 36;       // row stride of the staged 32-column block of L (same reason)
constexpr int BT_SL = bt::THREADS / (32 * (BT_RC / 4));   // row slices of the backward update

// Shared memory of the refine kernel, in this order: y (TL, nmax x BT_YS: the right-hand sides
// being solved), x (FP64, nmax x BT_RC: the solutions), Ls (TL, nmax x BT_LS: one staged block
// column of L, also the scratch of the permutations), the backward partial sums (TL,
// BT_SL x 32 x BT_RC), D^{-1} (2 x nmax TL and nmax kind bytes), per-column maxima (2 x BT_RC).
template <typename TL>
__host__ __device__ inline size_t bt_refine_bytes(int nmax) {
    const size_t ns = bt_stride(nmax);
    return ns * BT_YS * sizeof(TL) + ns * BT_RC * sizeof(double) + ns * BT_LS * sizeof(TL) +
           (size_t)BT_SL * 32 * BT_RC * sizeof(TL) + 2 * ns * sizeof(TL) + ns + 2 * BT_RC * sizeof(double) + 16;
}

template <typename TL>
size_t batched_refine_smem(int nrhs, int nmax) {
    (void)nrhs;
    return bt_refine_bytes<TL>(nmax);
}

// D^{-1} of the block-diagonal D, inverted in FP64 and rounded to TL: kind[i] = 0 for a 1x1
// block (y_i <- e_i y_i), 1 and 2 for the first and second position of a 2x2 block, whose
// inverse is [[e_i, f_i], [f_i, e_{i+1}]].  The 2x2 inverse uses the scaled form
// D = b [[a/b, 1], [1, c/b]], D^{-1} = [[c/b, -1], [-1, a/b]] / (b ((a/b)(c/b) - 1)).
template <typename TL>
__device__ void bt_dinv(int n, const double *Dd, const double *Ds, TL *e, TL *f, unsigned char *kind) {
    for (int i = threadIdx.x; i < n; i += bt::THREADS) {
        e[i] = TL(0);
        f[i] = TL(0);
        kind[i] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += bt::THREADS) {
        if (i > 0 && Ds[i - 1] != 0.0) continue;
        if (i + 1 < n && Ds[i] != 0.0) {
            const double bb = Ds[i], aa = Dd[i] / bb, cc = Dd[i + 1] / bb, den = bb * (aa * cc - 1.0);
            e[i] = (TL)(cc / den);
            e[i + 1] = (TL)(aa / den);
            f[i] = (TL)(-1.0 / den);
            f[i + 1] = TL(0);
            kind[i] = 1;
            kind[i + 1] = 2;
        } else {
            e[i] = (TL)(Dd[i] != 0.0 ? 1.0 / Dd[i] : 0.0);   // zero 1x1 block: pseudo-inverse 0
            f[i] = TL(0);
            kind[i] = 0;
        }
    }
}

// Stage the block column L(j0:n, j0:j0+nb) into Ls (row r - j0, column jj), strictly lower part
// of the diagonal block only (the unit diagonal is implicit), zeros elsewhere.
template <typename TL>
__device__ __forceinline__ void bt_stage(int n, int j0, int nb, const TL *L, int lda, TL *Ls) {
    const int rows = n - j0;
    for (int e = threadIdx.x; e < rows * 32; e += bt::THREADS) {
        const int r = e % rows, jj = e / rows;
        TL v = TL(0);
        if (jj < nb && r > jj) v = L[(size_t)(j0 + r) + (size_t)(j0 + jj) * lda];
        Ls[(size_t)r * BT_LS + jj] = v;
    }
}

// Bring the next block column of L (rows j0.. of columns j0 .. j0+31) towards L2 while the current
// one is being used: one prefetch per 128-byte line, so that the next staging does not wait for DRAM.
template <typename TL>
__device__ __forceinline__ void bt_prefetch_block(int n, int j0, const TL *L, int lda) {
    if (j0 < 0 || j0 >= n) return;
    const int nb = min(32, n - j0), rows = n - j0;
    constexpr int PER = 128 / (int)sizeof(TL);   // entries per line
    const int lines = (rows + PER - 1) / PER;
    for (int e = threadIdx.x; e < nb * lines; e += bt::THREADS) {
        const int c = e / lines, l = e % lines;
        const TL *a = L + (size_t)(j0 + l * PER) + (size_t)(j0 + c) * lda;
        asm volatile("prefetch.global.L2 [%0];" :: "l"(a));
    }
}

// y (n x rc, row stride BT_YS) <- (P L D L^T P^T)^{-1} y, by 32-column blocks of L staged in Ls.
template <typename TL>
__device__ void bt_solve(int n, int rc, const TL *L, int lda, const TL *de, const TL *df, const unsigned char *kind,
                         const int *perm, TL *y, TL *Ls, TL *part) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = (rc + 3) >> 2;
    bt_prefetch_block<TL>(n, 0, L, lda);   // the forward pass's first block column
    // v = P^T y: perm comes from the factor kernel; an index outside [0, n) (a factor that
    // never ran) is replaced so that no access leaves the system's rows
    for (int e = tid; e < n * BT_RC; e += bt::THREADS) {
        const int i = e / BT_RC, c = e % BT_RC;
        const int p = (unsigned)perm[i] < (unsigned)n ? perm[i] : i;
        Ls[(size_t)i * BT_YS + c] = y[(size_t)p * BT_YS + c];
    }
    __syncthreads();
    for (int e = tid; e < n * BT_RC; e += bt::THREADS) {
        const int i = e / BT_RC, c = e % BT_RC;
        y[(size_t)i * BT_YS + c] = Ls[(size_t)i * BT_YS + c];
    }
    // ---- forward: L v = v ----
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int nb = min(32, n - j0), rows = n - j0;
        __syncthreads();
        bt_stage<TL>(n, j0, nb, L, lda, Ls);
        bt_prefetch_block<TL>(n, j0 + 32, L, lda);
        __syncthreads();
        // the diagonal block, one warp per right-hand side, row = lane
        for (int c = warp; c < rc; c += bt::WARPS) {
            TL lrow[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) lrow[q] = lane < nb ? Ls[(size_t)lane * BT_LS + q] : TL(0);
            TL v = lane < nb ? y[(size_t)(j0 + lane) * BT_YS + c] : TL(0);
#pragma unroll
            for (int q = 0; q < 31; ++q) v -= lrow[q] * __shfl_sync(bt::FULLM, v, q);
            if (lane < nb) y[(size_t)(j0 + lane) * BT_YS + c] = v;
        }
        __syncthreads();
        // the rows below: y(r, :) -= L(r, B) y(B, :), 4 right-hand sides per task
        const int R = rows - nb;
        for (int e = tid; e < R * G; e += bt::THREADS) {
            const int r = nb + e % R, g = e / R;
            TL acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = y[(size_t)(j0 + r) * BT_YS + 4 * g + u];
            const TL *lr = Ls + (size_t)r * BT_LS;
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                const TL l = lr[q];
                const TL *yq = y + (size_t)(j0 + q) * BT_YS + 4 * g;
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] -= l * yq[u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) y[(size_t)(j0 + r) * BT_YS + 4 * g + u] = acc[u];
        }
    }
    __syncthreads();
    bt_prefetch_block<TL>(n, ((n - 1) / 32) * 32, L, lda);   // the backward pass's first block column
    // ---- block diagonal: v <- D^{-1} v ----
    for (int e = tid; e < n * rc; e += bt::THREADS) {
        const int i = e / rc, c = e % rc;
        const int kd = kind[i];
        if (kd == 0) {
            y[(size_t)i * BT_YS + c] *= de[i];
        } else if (kd == 1) {
            const TL y1 = y[(size_t)i * BT_YS + c], y2 = y[(size_t)(i + 1) * BT_YS + c];
            y[(size_t)i * BT_YS + c] = de[i] * y1 + df[i] * y2;
            y[(size_t)(i + 1) * BT_YS + c] = df[i] * y1 + de[i + 1] * y2;
        }
    }
    // ---- backward: L^T v = v, blocks from the bottom ----
    for (int j0 = ((n - 1) / 32) * 32; j0 >= 0; j0 -= 32) {
        const int nb = min(32, n - j0), rows = n - j0, R = rows - nb;
        __syncthreads();
        bt_stage<TL>(n, j0, nb, L, lda, Ls);
        bt_prefetch_block<TL>(n, j0 - 32, L, lda);
        __syncthreads();
        if (R > 0) {
            // y(B, :) -= L(below, B)^T y(below, :): BT_SL row slices, reduced after
            for (int e = tid; e < 32 * G * BT_SL; e += bt::THREADS) {
                const int jj = e & 31, g = (e >> 5) % G, sl = (e >> 5) / G;
                TL acc[4] = {TL(0), TL(0), TL(0), TL(0)};
                for (int r = nb + sl; r < rows; r += BT_SL) {
                    const TL l = Ls[(size_t)r * BT_LS + jj];
                    const TL *yr = y + (size_t)(j0 + r) * BT_YS + 4 * g;
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[u] += l * yr[u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) part[((size_t)sl * 32 + jj) * BT_RC + 4 * g + u] = acc[u];
            }
            __syncthreads();
            for (int e = tid; e < 32 * rc; e += bt::THREADS) {
                const int jj = e / rc, c = e % rc;
                if (jj < nb) {
                    TL s = TL(0);
#pragma unroll
                    for (int sl = 0; sl < BT_SL; ++sl) s += part[((size_t)sl * 32 + jj) * BT_RC + c];
                    y[(size_t)(j0 + jj) * BT_YS + c] -= s;
                }
            }
            __syncthreads();
        }
        for (int c = warp; c < rc; c += bt::WARPS) {
            TL lcol[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) lcol[q] = q < nb ? Ls[(size_t)q * BT_LS + lane] : TL(0);
            TL v = lane < nb ? y[(size_t)(j0 + lane) * BT_YS + c] : TL(0);
#pragma unroll
            for (int q = 31; q > 0; --q) v -= lcol[q] * __shfl_sync(bt::FULLM, v, q);
            if (lane < nb) y[(size_t)(j0 + lane) * BT_YS + c] = v;
        }
    }
    __syncthreads();
    // y <- P v
    for (int e = tid; e < n * BT_RC; e += bt::THREADS) {
        const int i = e / BT_RC, c = e % BT_RC;
        const int p = (unsigned)perm[i] < (unsigned)n ? perm[i] : i;
        Ls[(size_t)p * BT_YS + c] = y[(size_t)i * BT_YS + c];
    }
    __syncthreads();
    for (int e = tid; e < n * BT_RC; e += bt::THREADS) {
        const int i = e / BT_RC, c = e % BT_RC;
        y[(size_t)i * BT_YS + c] = Ls[(size_t)i * BT_YS + c];
    }
    __syncthreads();
}

// r = b - A x (FP64) for RG right-hand sides per task; y <- r rounded to TL, and the
// per-column maxima of |r| and |x|
template <int RG, typename TL>
__device__ void bt_residual(int n, int rc, const double *A, int lda, const double *Bv, int ldb, int c0,
                            const double *x, TL *y, double *rmax, double *xmax) {
    const int groups = rc / RG;
    for (int task = threadIdx.x; task < n * groups; task += bt::THREADS) {
        const int row = task % n, g = task / n;
        double acc[RG];
#pragma unroll
        for (int q = 0; q < RG; ++q) acc[q] = Bv[(size_t)row + (size_t)(c0 + g * RG + q) * ldb];
        for (int j = 0; j < n; ++j) {
            const double av = j <= row ? A[(size_t)row + (size_t)j * lda] : A[(size_t)j + (size_t)row * lda];
            const double *xj = x + (size_t)j * BT_RC + g * RG;
#pragma unroll
            for (int q = 0; q < RG; ++q) acc[q] -= av * xj[q];
        }
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const int c = g * RG + q;
            y[(size_t)row * BT_YS + c] = (TL)acc[q];
            atomicMax(reinterpret_cast<unsigned long long *>(rmax + c), (unsigned long long)__double_as_longlong(fabs(acc[q])));
            atomicMax(reinterpret_cast<unsigned long long *>(xmax + c),
                      (unsigned long long)__double_as_longlong(fabs(x[(size_t)row * BT_RC + c])));
        }
    }
}

template <typename TL>
__device__ void bt_refine_one(const BtRefineArgs<TL> &a, int sys, unsigned char *raw, double *s_an) {
    const int n = a.n[sys], tid = threadIdx.x;
    const size_t ns = bt_stride(a.nmax);
    TL *y = reinterpret_cast<TL *>(raw);
    double *x = reinterpret_cast<double *>(y + ns * BT_YS);
    TL *Ls = reinterpret_cast<TL *>(x + ns * BT_RC);
    TL *part = Ls + ns * BT_LS;
    TL *de = part + (size_t)BT_SL * 32 * BT_RC;
    TL *df = de + ns;
    double *rmax = reinterpret_cast<double *>(df + ns);
    double *xmax = rmax + BT_RC;
    unsigned char *kind = reinterpret_cast<unsigned char *>(xmax + BT_RC);
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
    const int *perm = a.perm[sys];
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
    }
    bt_dinv<TL>(n, a.Dd[sys], a.Ds[sys], de, df, kind);
    __syncthreads();
    const double an = A64 ? *s_an : 0.0;
    double worst = 0.0;
    int most = 0;
    for (int c0 = 0; c0 < a.nrhs; c0 += BT_RC) {
        const int rc = min(BT_RC, a.nrhs - c0);
        for (int e = tid; e < n * BT_RC; e += bt::THREADS) {
            const int i = e / BT_RC, c = e % BT_RC;
            y[(size_t)i * BT_YS + c] = c < rc ? (TL)Bv[(size_t)i + (size_t)(c0 + c) * ldb] : TL(0);
        }
        __syncthreads();
        bt_solve<TL>(n, rc, L, ldl, de, df, kind, perm, y, Ls, part);
        for (int e = tid; e < n * BT_RC; e += bt::THREADS) {
            const int i = e / BT_RC, c = e % BT_RC;
            x[(size_t)i * BT_RC + c] = (double)y[(size_t)i * BT_YS + c];
        }
        __syncthreads();
        int it = 0;
        double be = 0.0;
        while (A64) {
            for (int c = tid; c < BT_RC; c += bt::THREADS) { rmax[c] = 0.0; xmax[c] = 0.0; }
            __syncthreads();
            // rows x groups of right-hand sides: enough tasks for the CTA even for small n
            int rg = rc;
            while (rg > 1 && n * (rc / rg) < bt::THREADS && (rg & 1) == 0) rg >>= 1;
            if (rg != 16 && rg != 8 && rg != 4 && rg != 2) rg = 1;
            switch (rg) {
                case 16: bt_residual<16, TL>(n, rc, A64, lda64, Bv, ldb, c0, x, y, rmax, xmax); break;
                case 8: bt_residual<8, TL>(n, rc, A64, lda64, Bv, ldb, c0, x, y, rmax, xmax); break;
                case 4: bt_residual<4, TL>(n, rc, A64, lda64, Bv, ldb, c0, x, y, rmax, xmax); break;
                case 2: bt_residual<2, TL>(n, rc, A64, lda64, Bv, ldb, c0, x, y, rmax, xmax); break;
                default: bt_residual<1, TL>(n, rc, A64, lda64, Bv, ldb, c0, x, y, rmax, xmax); break;
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
            bt_solve<TL>(n, rc, L, ldl, de, df, kind, perm, y, Ls, part);
            for (int e = tid; e < n * rc; e += bt::THREADS) {
                const int i = e / rc, c = e % rc;
                x[(size_t)i * BT_RC + c] += (double)y[(size_t)i * BT_YS + c];
            }
            __syncthreads();
        }
        for (int e = tid; e < n * rc; e += bt::THREADS) {
            const int i = e % n, c = e / n;
            X[(size_t)i + (size_t)(c0 + c) * ldx] = x[(size_t)i * BT_RC + c];
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
// above[v] (v = 0..nmax, when given) = the number of systems with n > v: order[0 .. above[v])
// are those systems, order[above[v] .. batch) the others.
__global__ void batched_order_kernel(int batch, int nmax, const int *n, int *order, int *above) {
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
    // cnt[u] now counts the systems with nmax - n < u, i.e. n > nmax - u
    if (above)
        for (int v = threadIdx.x; v <= nmax; v += blockDim.x) above[v] = cnt[nmax - v];
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

cudaError_t launch_batched_order(int batch, int nmax, const int *n, int *order, int *above, cudaStream_t s) {
    batched_order_kernel<<<1, 1024, (size_t)(nmax + 1) * sizeof(int), s>>>(batch, nmax, n, order, above);
    count_launches(1);
    return cudaGetLastError();
}

size_t batched_max_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v > 1024 ? (size_t)v - 1024 : 0;   // room for the kernels' static shared memory
}

// the factor kernel for a shape and CTA size: the register sketch when it fits (FP32, d <= 48,
// nmax <= threads)
constexpr int BT_DR = 48;
template <typename T>
static void (*bt_factor_fn(int d, int nmax, int nt))(BtFactorArgs<T>) {
    if constexpr (sizeof(T) == 4) {
        if (bt_stride(d) <= BT_DR && nmax <= nt)
            return nt == 128 ? batched_factor_kernel<T, BT_DR, 128>
                 : nt == 256 ? batched_factor_kernel<T, BT_DR, 256> : batched_factor_kernel<T, BT_DR, 512>;
    }
    (void)d;
    (void)nmax;
    return nt == 128 ? batched_factor_kernel<T, 0, 128>
         : nt == 256 ? batched_factor_kernel<T, 0, 256> : batched_factor_kernel<T, 0, 512>;
}

template <typename T>
int batched_factor_grid(int d, int b, int nmax, int nt) {
    if (nt != 128 && nt != 256 && nt != 512) return 0;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = batched_factor_smem<T>(d, b, nmax);
    void (*fn)(BtFactorArgs<T>) = bt_factor_fn<T>(d, nmax, nt);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, nt, smem);
    return sms * (per > 0 ? per : 1);
}

template <typename T>
cudaError_t launch_batched_factor(int batch, int d, int b, int nmax, const int *n, const double *const *A64,
                                  const int *lda64, T *const *A, const int *lda, double *const *Dd, double *const *Ds,
                                  int *const *perm, const T *om, double alpha, int *info, const int *order,
                                  int *ticket, int *pscr, int grid, int nt, const int *first, const int *last,
                                  cudaStream_t s) {
    if (nt != 128 && nt != 256 && nt != 512) return cudaErrorInvalidValue;
    BtFactorArgs<T> a{batch, d, b, nmax, n, A64, lda64, A, lda, Dd, Ds, perm, om, alpha, info, order, ticket, pscr,
                      first, last};
    const size_t smem = batched_factor_smem<T>(d, b, nmax);
    void (*fn)(BtFactorArgs<T>) = bt_factor_fn<T>(d, nmax, nt);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ticket, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    fn<<<grid < batch ? grid : batch, nt, smem, s>>>(a);
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
    template int batched_factor_grid<T>(int, int, int, int);                                                         \
    template cudaError_t launch_batched_factor<T>(int, int, int, int, const int *, const double *const *, const int *, \
                                                  T *const *, const int *, double *const *, double *const *,          \
                                                  int *const *, const T *, double, int *, const int *, int *, int *,  \
                                                  int, int, const int *, const int *, cudaStream_t);                 \
    template cudaError_t launch_batched_refine<T>(int, int, int, int, double, const int *, const T *const *,          \
                                                  const int *, const double *const *, const double *const *,          \
                                                  const int *const *, const double *const *, const int *,             \
                                                  const double *const *, const int *, double *const *, const int *,   \
                                                  double *, int *, const int *, int *, cudaStream_t);
BT_INST(float)
BT_INST(double)
#undef BT_INST

}  // namespace rcpk
