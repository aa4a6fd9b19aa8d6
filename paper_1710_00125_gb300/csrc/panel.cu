// panel.cu -- one panel of Algorithm 1 (q = 1) as a persistent cooperative kernel.
//
// Each launch performs up to b pivot steps starting at column k0 (read from the device
// state), on the matrix in "block-start" order: every earlier panel's interchanges and
// trailing update are already applied.  Ownership is by block-start index: CTA c owns the
// indices [k0 + c*chunk, k0 + (c+1)*chunk) and keeps, in shared memory, their sketch
// columns B(:, j), their rows of W = L D for this panel's columns, and the current diagonal
// of the Schur complement.  An interchange therefore moves no data during the panel; it only
// relabels positions (lp[] per owned index, and a small window table of which index sits at
// the positions k0 .. k0+b+2 the panel can fill).  The data are moved once per panel by the
// interchange kernels (interchange.cu).  With the Algorithm 2 safeguard on, a step whose
// pivot's sketch norm falls below eps^delta beta ends the panel before that step, and the host
// recomputes the sketch or stops.
//
// Per pivot step (Section 3, Figure SBKP, Eq. "Update matrix B"):
//   (1) argmax of ||B(:, j)||^2 over the remaining indices (ties: smallest position)  -> P
//       grid barrier #1
//   (2) the interchange k <-> position(P); column P of the Schur complement,
//       c_j = A(j, P) - sum_t W(j, t) L(P, t) (a GEMV over the panel built so far);
//       lambda = max_{j != P} |c_j| at r (ties: smallest position)
//       grid barrier #2
//   (3) SBKP case (0)-(3) with alpha; for cases (2)/(3) column r of the Schur complement
//   (4) multipliers (1x1: c / a_kk; 2x2: [c_j c'_j] D_k^{-1}, its scalars in FP64), W = L D,
//       the Schur diagonal update, and the rank-s sketch update fused with the next norms.
// Grid-wide argmax: in FP32 every CTA folds its candidate into one 64-bit word with red.max
// (value bits | inverted position | index), so a reader needs a single L2 load; in FP64 the
// value does not fit beside the position, so every CTA publishes a record and the readers
// reduce all records.  The winner's scalars and sketch column are fetched together with the
// column of A they select, so each barrier is followed by one dependent L2 and one HBM trip.
#include <climits>
#include <type_traits>

#include "kernels.h"

namespace rcpk {

constexpr int PANEL_THREADS = 512;
constexpr int PANEL_WARPS = PANEL_THREADS / 32;
constexpr unsigned FULL = 0xffffffffu;

// Row strides of the per-row shared arrays: a quad of threads works on one row and walks the
// row with stride 4, so a stride of 4 (mod 32) words puts the 8 rows x 4 threads of a warp on
// 32 different banks.
__host__ __device__ constexpr int quad_stride(int x) { return x + ((36 - (x % 32)) % 32); }

template <typename T>
size_t panel_smem_bytes(int d, int bw, int chunk_cap, int spec) {
    size_t s = 0;
    if (spec == 1) s += (size_t)chunk_cap * (quad_stride(d) + 1) * sizeof(T) + 16;   // shadow sketch + norms
    if (spec == 2) s += ((size_t)2 * chunk_cap + d) * sizeof(T) + 16;   // deferred: norms, multipliers, pivot column
    s += (size_t)chunk_cap * sizeof(double);           // nrm (T, padded to 8 bytes)
    s += (size_t)chunk_cap * quad_stride(d) * sizeof(T);    // Bs
    s += (size_t)chunk_cap * quad_stride(bw) * sizeof(T);   // Ws
    s += (size_t)chunk_cap * 5 * sizeof(T);            // dg, c1, c2, l1s, l2s
    s += (size_t)2 * d * sizeof(T);                    // bP, bR
    s += (size_t)2 * bw * sizeof(T);                   // lP, lR
    s += (size_t)4 * bw * sizeof(T) + (size_t)bw * sizeof(int);   // per-column D scalars and kinds
    s += (size_t)chunk_cap * 2 * sizeof(int);          // lp, alive
    s += (size_t)(bw + 3) * sizeof(int);               // window (kinds counted above)
    return s + 64;
}

template <typename V>
struct CandT {
    V v;
    int lpos;
    int phys;
};
using Cand = CandT<double>;

template <typename V>
__device__ __forceinline__ bool better(V v1, int l1, V v2, int l2) {
    return v1 > v2 || (v1 == v2 && l1 < l2);
}

template <typename V>
__device__ __forceinline__ CandT<V> warp_argmax(CandT<V> c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        V v = __shfl_down_sync(FULL, c.v, off);
        int l = __shfl_down_sync(FULL, c.lpos, off);
        int p = __shfl_down_sync(FULL, c.phys, off);
        if (better(v, l, c.v, c.lpos)) { c.v = v; c.lpos = l; c.phys = p; }
    }
    return c;
}

// Block-wide argmax; the result is returned to every thread.
template <typename V>
__device__ __forceinline__ CandT<V> block_argmax(CandT<V> c, CandT<V> *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    c = warp_argmax(c);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    if (warp == 0) {
        CandT<V> x = lane < PANEL_WARPS ? red[lane] : CandT<V>{V(-1), INT_MAX, -1};
        x = warp_argmax(x);
        if (lane == 0) red[PANEL_WARPS] = x;
    }
    __syncthreads();
    CandT<V> r = red[PANEL_WARPS];
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T s) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
    return s;
}

template <typename T>
__device__ __forceinline__ T a_sym(const T *__restrict__ A, int lda, int i, int j) {
    return i >= j ? A[(size_t)i + (size_t)j * lda] : A[(size_t)j + (size_t)i * lda];
}

// Reduction slots: one 32-byte record per CTA {value, aux1, aux2, (position, index)}.
__device__ __forceinline__ void slot_write(double *slots, int cta, double v, double a1, double a2, int lpos, int phys) {
    double2 *p = reinterpret_cast<double2 *>(slots + 4 * (size_t)cta);
    unsigned long long packed = ((unsigned long long)(unsigned)phys << 32) | (unsigned)lpos;
    __stcg(p, make_double2(v, a1));
    __stcg(p + 1, make_double2(a2, __longlong_as_double((long long)packed)));
}

struct SlotWin {
    double v, a1, a2;
    int lpos, phys, cta;
};

// Warp 0: reads all G records in one pass and returns the best (value desc, position asc).
__device__ __forceinline__ SlotWin slot_reduce(const double *slots, int G) {
    const int lane = threadIdx.x & 31;
    SlotWin b{-1.0, 0.0, 0.0, INT_MAX, -1, -1};
    for (int g = lane; g < G; g += 32) {
        const double2 *p = reinterpret_cast<const double2 *>(slots + 4 * (size_t)g);
        double2 x = __ldcg(p), y = __ldcg(p + 1);
        unsigned long long packed = (unsigned long long)__double_as_longlong(y.y);
        int lpos = (int)(unsigned)(packed & 0xffffffffull), phys = (int)(unsigned)(packed >> 32);
        if (better(x.x, lpos, b.v, b.lpos)) b = SlotWin{x.x, x.y, y.x, lpos, phys, g};
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        SlotWin o;
        o.v = __shfl_down_sync(FULL, b.v, off);
        o.a1 = __shfl_down_sync(FULL, b.a1, off);
        o.a2 = __shfl_down_sync(FULL, b.a2, off);
        o.lpos = __shfl_down_sync(FULL, b.lpos, off);
        o.phys = __shfl_down_sync(FULL, b.phys, off);
        o.cta = __shfl_down_sync(FULL, b.cta, off);
        if (better(o.v, o.lpos, b.v, b.lpos)) b = o;
    }
    return b;   // valid in lane 0
}

static_assert(2 * KEY_RING * KEY_STRIDE <= PANEL_KEY_WORDS, "the pivot and speculative key rings");

// Block-wide maximum of two packed keys per thread (the result to every thread): per warp two
// 32-bit redux.sync per key (high word, then the low word among the lanes holding the maximal
// high word), one shared slot per key and warp, and the same warp reduction over the slots.
// Two slot sets are used in alternation (call counter `cnt`, uniform over the block): the set
// of call c is rewritten at call c + 2, after the CTA barrier of call c + 1.
constexpr int RED2_SLOTS = 4 * (PANEL_THREADS / 32);   // [2 sets][2 keys][warps]

__device__ __forceinline__ void block_max2_u64(unsigned long long &a, unsigned long long &b, unsigned long long *red,
                                               int &cnt) {
    constexpr int W = PANEL_THREADS / 32;
    static_assert(W <= 32, "one warp reduces the per-warp slots");
    const unsigned long long wa = warp_max_u64(a), wb = warp_max_u64(b);
    unsigned long long *set = red + (cnt & 1) * 2 * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        set[warp] = wa;
        set[W + warp] = wb;
    }
    __syncthreads();
    a = warp_max_u64(lane < W ? set[lane] : 0ull);
    b = warp_max_u64(lane < W ? set[W + lane] : 0ull);
    ++cnt;
}

// The multiplier L(j, t) of a row from its W = L D row and the panel's per-column D scalars,
// with the same operations the elimination used (so the result is bitwise the same): kind 0
// (zero column), 1 (1x1: w / d, or w * (1/d) in FP32), 3 / 4 (first / second column of a 2x2
// block: scaled inverse).
template <typename T>
__device__ __forceinline__ T l_entry(const T *wr, int t, const int *kind, const T *cs0, const T *cs1, const T *cs2,
                                     const T *cs3) {
    constexpr bool F64 = std::is_same<T, double>::value;
    const int k = kind[t];
    if (k == 1) return F64 ? wr[t] / cs0[t] : wr[t] * cs0[t];
    if (k == 3 || k == 4) {
        const int t0 = k == 3 ? t : t - 1;
        const T r = cs3[t0];
        const T x1 = F64 ? wr[t0] / r : wr[t0] * r, x2 = F64 ? wr[t0 + 1] / r : wr[t0 + 1] * r;
        return k == 3 ? cs2[t0] * (cs1[t0] * x1 - x2) : cs2[t0] * (cs0[t0] * x2 - x1);
    }
    return T(0);
}

// c[jl] = A(j, X) - sum_{t < i} Ws[jl][t] L(X, t) for the alive owned rows.  The loads of
// the column of A, of the candidate's sketch column (into bX), of its multiplier row L(X, 0:i)
// (into lX) and of `nx` scalars of the candidate's slot (into xs, thread 0) are all issued
// before the first barrier so that their latencies overlap.  `hook` runs on thread 0 right
// after that barrier.
template <typename T, typename Hook>
__device__ void schur_column(const T *__restrict__ A, int lda, int j_lo, int cnt, int X, int i, int bw,
                             const T *Ws, const T *payg, T *bX, const T *lXg, T *lX, int d,
                             const int *alive, T *c, const T *xsrc, T *xs, int nx, Hook hook,
                             bool preloaded = false, T pa0 = T(0), T pa1 = T(0)) {
    T a0 = pa0, a1 = pa1;
    const int r0 = threadIdx.x, r1 = threadIdx.x + PANEL_THREADS;
    if (!preloaded) {   // else the caller already has the column in (pa0, pa1) and bX, lX, xs filled
        if (r0 < cnt && alive[r0]) a0 = a_sym(A, lda, j_lo + r0, X);
        if (r1 < cnt && alive[r1]) a1 = a_sym(A, lda, j_lo + r1, X);
        for (int r = threadIdx.x; r < d; r += PANEL_THREADS) bX[r] = ldcg(payg + r);
        for (int t = threadIdx.x; t < i; t += PANEL_THREADS) lX[t] = ldcg(lXg + t);
        if (threadIdx.x < nx) xs[threadIdx.x] = ldcg(xsrc + threadIdx.x);
    }
    __syncthreads();
    if (threadIdx.x == 0) hook();
    // four threads per row, each summing every fourth term, combined by two shuffles
    const int sub = threadIdx.x & 3;
    for (int jl0 = 0; jl0 < cnt; jl0 += PANEL_THREADS / 4) {
        const int jl = jl0 + (threadIdx.x >> 2);
        T s = T(0);
        if (jl < cnt && alive[jl] && i > 0) {
            const T *wr = Ws + (size_t)jl * bw;
            for (int t = sub; t < i; t += 4) s = fma(wr[t], lX[t], s);
        }
        s += __shfl_xor_sync(FULL, s, 1);
        s += __shfl_xor_sync(FULL, s, 2);
        if (sub == 0 && jl < cnt) c[jl] = s;
    }
    __syncthreads();
    if (r0 < cnt) c[r0] = alive[r0] ? (T)(a0 - c[r0]) : T(0);
    if (r1 < cnt) c[r1] = alive[r1] ? (T)(a1 - c[r1]) : T(0);
    __syncthreads();
}

// A(j, X) for the owned row that the fused FP32 step assigns to this thread's register m:
// row q + 128 (s + 4 m) for quad q and quad lane s (0 for dead rows and for index `skip`).
template <typename T>
__device__ __forceinline__ T a_quad(const T *__restrict__ A, int lda, int j_lo, int cnt, const int *alive, int X,
                                    int m, int skip) {
    const int jl = (threadIdx.x >> 2) + (PANEL_THREADS / 4) * ((threadIdx.x & 3) + 4 * m);
    return (jl < cnt && alive[jl] && j_lo + jl != skip) ? a_sym(A, lda, j_lo + jl, X) : T(0);
}

struct NoHook {
    __device__ void operator()() const {}
};

// correctly rounded reciprocal in the factor's type
__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_rn(double x) { return 1.0 / x; }

constexpr int CASE_PENDING = 4;   // lambda > 0 and |a_kk| < alpha lambda: case 2 or 3, a_rr needed

// SBKP decision and the per-step scalars (thread 0).  FP64 arithmetic; the FP32 path uses
// one reciprocal of the off-diagonal entry instead of two divisions.
template <typename T>
__device__ void sbkp_scalars(int kase, double akk, double lam, double ark, double arr, double alpha, int *s_i,
                             double *s_d, T *s_t, T rkk) {
    if (kase == CASE_PENDING) {
        if (!isfinite(ark) || !isfinite(arr)) kase = -1;
        else kase = fabs(arr) >= alpha * lam ? 2 : 3;
    }
    s_i[7] = kase;
    const double dpiv = kase == 2 ? arr : akk;
    s_d[3] = ark;
    s_d[4] = arr;
    s_d[5] = dpiv;
    if (kase == 3) {
        double aa, cc, r;
        if (std::is_same<T, double>::value) { aa = akk / ark; cc = arr / ark; r = 1.0 / ark; }
        else { r = 1.0 / ark; aa = akk * r; cc = arr * r; }
        const double tinv = 1.0 / (aa * cc - 1.0);
        s_t[0] = (T)aa; s_t[1] = (T)cc; s_t[2] = (T)tinv; s_t[3] = (T)ark; s_t[4] = (T)r;
    } else {
        s_t[0] = s_t[1] = s_t[2] = T(0);
        s_t[3] = T(1); s_t[4] = T(1);
    }
    s_t[5] = (T)dpiv;
    s_t[6] = kase == 1 ? rkk : (kase == 2 ? (T)(1.0 / dpiv) : T(0));
    s_i[8] = dpiv != 0.0;
}

// DEF: the speculative sketch update is deferred to the next step's pass (w.spec == 2, FP32 only);
// a separate instantiation, so that the shadow-copy kernel carries none of its code.
template <typename T, bool DEF>
__global__ void __launch_bounds__(PANEL_THREADS, 1) panel_kernel(FactorWork<T> w) {
    constexpr bool KEYS = std::is_same<T, float>::value;   // packed-key argmax (FP32 values)
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ CandT<T> s_red[PANEL_WARPS + 1];
    __shared__ int s_i[16];
    __shared__ double s_d[16];
    __shared__ T s_t[8];
    __shared__ T s_x[16];   // per-step scalars in the factor's type: [0] pivot norm, [2] lambda,
                            // [6] next pivot norm (speculation), [8] a_kk, [10..11] a_rk, a_rr
    __shared__ unsigned long long s_red2[RED2_SLOTS];

    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (ldcg(w.status) != 0) return;
    const int n = w.n, d = w.d, bw = w.bw, lda = w.lda;
    const int k0 = ldcg(&w.st->next);
    if (k0 >= n) {
        // nothing left: record an empty panel so that the interchange and trailing kernels
        // of this round do nothing (they must not replay the previous panel's record)
        if (cta == 0 && tid == 0) {
            w.st->n_moved = 0;
            w.st->k0 = n;
            w.st->kend = n;
        }
        return;
    }
    const int m = n - k0;
    const int chunk = (m + G - 1) / G;
    if (chunk > w.chunk_cap || chunk > 2 * PANEL_THREADS) {
        if (tid == 0) atomicOr(w.status, ST_INTERNAL);
        return;
    }
    const int j_lo = k0 + cta * chunk;
    const int cnt = max(0, min(n, j_lo + chunk) - j_lo);
    const int cap = w.chunk_cap;

    const int ds = quad_stride(d), ws = quad_stride(bw);   // shared-memory row strides
    T *nrm = reinterpret_cast<T *>(smem);
    T *Bs = reinterpret_cast<T *>(reinterpret_cast<double *>(smem) + cap);   // swapped with Bs2 on a committed speculation
    T *Ws = Bs + (size_t)cap * ds;
    T *dg = Ws + (size_t)cap * ws;
    T *c1 = dg + cap;
    T *c2 = c1 + cap;
    T *dg2 = c2 + cap;                 // shadow diagonal of the speculative case-(1) elimination
    T *bP = c2 + 3 * (size_t)cap;      // (one spare row kept for alignment of the layout)
    T *bR = bP + d;
    T *lP = bR + d;
    T *lR = lP + bw;
    T *cs0 = lR + bw, *cs1 = cs0 + bw, *cs2 = cs1 + bw, *cs3 = cs2 + bw;   // per-column D scalars
    int *lp = reinterpret_cast<int *>(cs3 + bw);
    int *alive = lp + cap;
    int *win = alive + cap;           // positions k0 .. k0 + bw + 2
    int *ckind = win + (bw + 3);      // per panel column: 0 zero, 1 scalar, 3/4 first/second of 2x2
    // shadow sketch columns and norms for the speculative case-(1) update (when w.spec)
    // shadow sketch columns and norms for the speculative case-(1) update (w.spec == 1), or, when
    // the shadow does not fit (w.spec == 2, deferred), only the norms, each row's multiplier of the
    // speculative update (l1s) and the pivot's sketch column of a confirmed update not yet applied
    T *Bs2 = reinterpret_cast<T *>(ckind + bw);
    T *nrm2 = Bs2 + (w.spec == 1 ? (size_t)cap * ds : 0);
    T *l1s = nrm2 + cap;
    T *bPd = l1s + cap;
    constexpr bool deferred = KEYS && DEF;
    bool pend = false;   // deferred: a confirmed speculative sketch update (bPd, l1s) awaits the next pass
    const int wsz = bw + 3;

    const T *__restrict__ A = w.A;
    // optional per-step timestamps of CTA 0 (profiling only)
    unsigned long long *const trace = (cta == 0 && tid == 0) ? w.trace : nullptr;
#define PANEL_MARK(slot) \
    do { if (trace) trace[(size_t)k * PANEL_TRACE_SLOTS + (slot)] = clock64(); } while (0)
    // ---- load the owned state ----
    for (int e = tid; e < cnt * d; e += PANEL_THREADS) {
        int jl = e / d, r = e - jl * d;
        Bs[(size_t)jl * ds + r] = w.B[(size_t)r + (size_t)(j_lo + jl) * d];
    }
    for (int e = tid; e < cnt * ws; e += PANEL_THREADS) Ws[e] = T(0);
    for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
        int j = j_lo + jl;
        dg[jl] = A[(size_t)j + (size_t)j * lda];
        lp[jl] = j;
        alive[jl] = 1;
    }
    for (int x = tid; x < wsz; x += PANEL_THREADS) win[x] = k0 + x;
    double beta2 = 0.0;   // thread 0 of CTA 0: ||B^(1)||_{1,2}^2
    if (tid == 0) {
        s_i[0] = (int)barrier_base(w.bar, (unsigned)G);
        if (cta == 0) {
            w.st->n_moved = 0;
            beta2 = ldcg(&w.st->beta2);
            // panel maxima, raised by every CTA's epilogue (after at least one grid barrier)
            w.st->tcW_bits = 0ull;
            w.st->tcL_bits = 0ull;
        }
    }
    __syncthreads();
    // initial column norms
    for (int jl = warp; jl < cnt; jl += PANEL_WARPS) {
        T s = T(0);
        for (int r = lane; r < d; r += 32) { T b = Bs[(size_t)jl * ds + r]; s = fma(b, b, s); }
        s = warp_sum(s);
        if (lane == 0) nrm[jl] = s;
    }
    const unsigned base = (unsigned)s_i[0];
    const unsigned gbase = base / (unsigned)G;   // barriers completed before this launch
    unsigned nbar = 0;
    int k = k0, i = 0, n2 = 0;
    double maxD = 0.0, minnorm2 = INFINITY;
    T maxDf = T(0), beta2f = T(0), minnorm2f = (T)INFINITY;   // FP32 path: the same, in the factor's type
    int red2_cnt = 0;   // calls of block_max2_u64 (slot rotation)
    T tmaxL = T(0);
    int info = 0, fail = 0;
    const double alpha = w.alpha;
    const int ps = d;        // payload record: the candidate's sketch column
    T *pay1 = w.pay, *pay2 = w.pay + (size_t)G * ps;
    double *rec1 = w.s1v, *rec2 = w.s2v;   // per-CTA records (4 doubles each)
    unsigned long long *keys = w.keys;
    // speculative case-(1) state (FP32 path with room for the shadow sketch)
    unsigned long long *spec_keys = (KEYS && w.spec) ? w.keys + KEY_RING * KEY_STRIDE : nullptr;
    T *spec_pay = w.pay + (size_t)2 * G * ps;                 // [2][G][d], by barrier parity
    double *spec_rec = w.s3v;                                  // [2][G][4]
    bool have_next = false;
    // Algorithm 2: the pivot's squared sketch norm against (eps^delta beta)^2 with
    // delta = (recomputations + 1) / r; beta^2 is the first pivot's squared norm
    double gfac = 0.0, gthr2 = 0.0;
    if (w.guard_r > 0) {
        gfac = pow(w.guard_eps, 2.0 * (double)(ldcg(&w.st->nresk) + 1) / (double)w.guard_r);
        gthr2 = ldcg(&w.st->beta2) * gfac;
    }
    int gstop = 0;
    int run1 = 2;   // consecutive case-(0)/(1) steps; speculate when >= 2
    T preA0 = T(0), preA1 = T(0);   // next pivot's column of A, loaded during a commit
    __syncthreads();

    while (i < w.bmax && k < n) {
        PANEL_MARK(0);
        // ---------------- (1) sketch column-norm argmax ----------------
        // (skipped when the previous step's speculation already found this step's pivot)
        if (!have_next) {
        CandT<T> c{T(-1), INT_MAX, -1};
        for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
            // q = b: the candidate is the column at position k (placed there by the block QRCP)
            const T v = w.qb ? (lp[jl] == k ? T(1) : T(-1)) : nrm[jl];
            if (alive[jl] && v >= T(0) && better(v, lp[jl], c.v, c.lpos)) c = CandT<T>{v, lp[jl], j_lo + jl};
        }
        c = block_argmax(c, s_red);
        if (c.phys >= 0) {
            const int jc = c.phys - j_lo;
            for (int r = tid; r < d; r += PANEL_THREADS) stcg(pay1 + (size_t)cta * ps + r, Bs[(size_t)jc * ds + r]);
        }
        const unsigned g1 = gbase + nbar + 1;
        if (tid == 0) {
            if (KEYS) {
                if (c.phys >= 0) {
                    stcg(reinterpret_cast<T *>(rec1 + 4 * (size_t)cta), dg[c.phys - j_lo]);
                    red_max_u64(key_slot(keys, g1), make_key((float)c.v, c.lpos, c.phys));
                }
            } else {
                const double dgc = c.phys >= 0 ? (double)dg[c.phys - j_lo] : 0.0;
                slot_write(rec1, cta, (double)c.v, dgc, 0.0, c.lpos, c.phys);
            }
        }
        PANEL_MARK(1);
        if (!grid_barrier(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
        PANEL_MARK(2);
        if (KEYS) {
            if (tid == 0) {
                const unsigned long long key = ld_key(key_slot(keys, g1));
                if (cta == 0) {
                    *key_slot(keys, g1 + KEY_RING / 2) = 0ull;
                    if (spec_keys) *key_slot(spec_keys, g1 + KEY_RING / 2) = 0ull;
                }
                if (key != 0ull) {
                    s_i[1] = (int)(key & 0xFFFFull);
                    s_i[2] = 0xFFFF - (int)((key >> 16) & 0xFFFFull);
                    s_i[3] = (s_i[1] - k0) / chunk;
                    s_x[0] = (T)__uint_as_float((unsigned)(key >> 32));
                } else {
                    s_i[1] = -1;
                }
            }
        } else if (warp == 0) {
            SlotWin b = slot_reduce(rec1, G);
            if (lane == 0) {
                s_i[1] = b.phys; s_i[2] = b.lpos; s_i[3] = b.cta;
                s_d[0] = b.v; s_d[1] = b.a1;
                s_x[0] = (T)b.v;
            }
        }
        if (tid == 0 && s_i[1] >= 0) {
            // interchange k <-> LP (positions); Q is the index now at position k
            const int P = s_i[1], LP = s_i[2];
            const int Q = win[k - k0];
            if (LP - k0 < wsz) win[LP - k0] = Q;
            win[k - k0] = P;
            if (P >= j_lo && P < j_lo + cnt) lp[P - j_lo] = k;
            if (Q != P && Q >= j_lo && Q < j_lo + cnt) lp[Q - j_lo] = LP;
            if (cta == 0 && !w.qb) {
                if (KEYS) {
                    if (k == 0) beta2f = s_x[0];
                    minnorm2f = fminf((float)minnorm2f, (float)s_x[0]);
                } else {
                    if (k == 0) { beta2 = s_d[0]; w.st->beta2 = beta2; }
                    minnorm2 = fmin(minnorm2, s_d[0]);
                }
            }
        }
        __syncthreads();
        }   // !have_next (a committed speculation did this step's interchange bookkeeping and
            // ended with a CTA barrier)
        const int P = s_i[1], gP = s_i[3];
        if (P < 0 || !isfinite(s_x[0])) { fail = ST_NONFINITE; break; }
        if (w.guard_r > 0) {
            // the panel ends before step k (whose interchange only permuted the unfactored
            // part); the host recomputes the sketch or stops
            const double t2 = (double)s_x[0];
            if (k > 0 && t2 < gthr2) { gstop = 1; break; }
            if (k == 0) gthr2 = t2 * gfac;
        }
        // where step (1) published P's sketch column and a_kk (read only without a committed
        // speculation, whose commit already loaded them)
        const T *payP = pay1 + (size_t)gP * ps;
        const T *recP = reinterpret_cast<const T *>(rec1 + 4 * (size_t)gP);

        // ---------------- (2) column P of the Schur complement, lambda and r ----------------
        PANEL_MARK(3);
        const unsigned g2 = gbase + nbar + 1;
        // speculation (FP32): assume case (1) (multipliers c / a_kk), update the sketch into the
        // shadow buffer and find the next step's pivot candidate before the barrier
        const bool spec = KEYS && spec_keys && run1 >= 2 && i + 1 < w.bmax && k + 1 < n;
        const int par = (int)(g2 & 1u);
        unsigned long long kl = 0ull, ks = 0ull;   // FP32: best lambda key, best speculative sketch key
        T akkT = T(0);                              // a_kk in the factor's type
        T fk = T(0);                                // FP32: its reciprocal (0 for a zero pivot)
        double akk = 0.0;                           // FP64 path: a_kk
        if (KEYS) {
            // One pass per quad of threads and owned row: the row's entry of column P of the
            // Schur complement, its lambda key and, when speculating, its case-(1) sketch update
            // and norm.  A(j, P) of row q + 128 m sits in quad lane m % 4, register m / 4.
            if (!have_next) {
                preA0 = a_quad<T>(A, lda, j_lo, cnt, alive, P, 0, -1);
                preA1 = a_quad<T>(A, lda, j_lo, cnt, alive, P, 1, -1);
                for (int r = tid; r < d; r += PANEL_THREADS) bP[r] = ldcg(payP + r);
                for (int t = tid; t < i; t += PANEL_THREADS) lP[t] = ldcg(w.Lg + (size_t)P * bw + t);
                if (tid == 0) s_x[8] = ldcg(recP);
                __syncthreads();
            }
            akkT = s_x[8];
            if (!isfinite(akkT)) { fail = ST_NONFINITE; break; }
            // reciprocal of a_kk (case (1) and the speculation), in every thread
            const T f = akkT != T(0) ? recip_rn(akkT) : T(0);
            fk = f;
            if (tid == 0) s_t[7] = f;
            PANEL_MARK(10);
            const int sub = tid & 3;
            for (int m = 0; m * (PANEL_THREADS / 4) < cnt; ++m) {
                const int jl = m * (PANEL_THREADS / 4) + (tid >> 2);
                const bool in = jl < cnt && alive[jl];
                T sdot = T(0);
                if (in && i > 0) {
                    const T *wr = Ws + (size_t)jl * ws;
                    for (int t = sub; t < i; t += 4) sdot = fma(wr[t], lP[t], sdot);
                }
                sdot += __shfl_xor_sync(FULL, sdot, 1);
                sdot += __shfl_xor_sync(FULL, sdot, 2);
                const T aj = __shfl_sync(FULL, (m >> 2) == 0 ? preA0 : preA1, (lane & ~3) | (m & 3));
                if (m == 0) PANEL_MARK(15);
                const T cv = in ? (T)(aj - sdot) : T(0);
                if (sub == 0 && jl < cnt) c1[jl] = cv;
                const bool live = in && j_lo + jl != P;
                T sacc = T(0);
                if (deferred) {
                    // the confirmed speculative update of the previous step, in place, on every live
                    // row (with the operations the shadow sketch uses), then this step's speculative
                    // update for its norm only; the row's multiplier is kept for the next pass
                    const bool app = pend && in, sp = spec && live;
                    const T l0 = app ? l1s[jl] : T(0);
                    const T l1 = cv * f;
                    __syncwarp();   // every lane of the quad has read l1s[jl] before it is rewritten
                    if (app || sp) {
                        T *col = Bs + (size_t)jl * ds;
                        for (int r0 = sub; r0 < d; r0 += 20) {
                            T v[5], pd[5], pb[5];
#pragma unroll
                            for (int q = 0; q < 5; ++q) {
                                const int r = r0 + 4 * q;
                                v[q] = r < d ? col[r] : T(0);
                                pd[q] = (app && r < d) ? bPd[r] : T(0);
                                pb[q] = (sp && r < d) ? bP[r] : T(0);
                            }
#pragma unroll
                            for (int q = 0; q < 5; ++q) {
                                const int r = r0 + 4 * q;
                                if (app) {
                                    v[q] = v[q] - pd[q] * l0;
                                    if (r < d) col[r] = v[q];
                                }
                                if (sp) {
                                    const T x = v[q] - pb[q] * l1;
                                    sacc = fma(x, x, sacc);
                                }
                            }
                        }
                    }
                    if (sp && sub == 0) l1s[jl] = l1;
                } else if (spec && live) {
                    const T l1 = cv * f;
                    const T *col = Bs + (size_t)jl * ds;
                    T *col2 = Bs2 + (size_t)jl * ds;
                    // rows sub, sub+4, ...: five at a time, all loads of a chunk before its
                    // stores (the sketch copies and the pivot column share one base)
                    for (int r0 = sub; r0 < d; r0 += 20) {
                        T v[5], pb[5];
#pragma unroll
                        for (int q = 0; q < 5; ++q) {
                            const int r = r0 + 4 * q;
                            v[q] = r < d ? col[r] : T(0);
                            pb[q] = r < d ? bP[r] : T(0);
                        }
#pragma unroll
                        for (int q = 0; q < 5; ++q) {
                            const int r = r0 + 4 * q;
                            const T x = v[q] - pb[q] * l1;
                            if (r < d) col2[r] = x;
                            sacc = fma(x, x, sacc);
                        }
                    }
                }
                if (spec) {
                    sacc += __shfl_xor_sync(FULL, sacc, 1);
                    sacc += __shfl_xor_sync(FULL, sacc, 2);
                }
                if (live && sub == 0) {
                    kl = max(kl, make_key((float)fabs(cv), lp[jl], j_lo + jl));
                    if (spec) {
                        nrm2[jl] = sacc;
                        ks = max(ks, make_key((float)sacc, lp[jl], j_lo + jl));
                    }
                }
            }
            pend = false;   // (deferred) applied to every live row above
        } else {
            schur_column<T>(A, lda, j_lo, cnt, P, i, ws, Ws, payP, bP, w.Lg + (size_t)P * bw, lP, d,
                            alive, c1, recP, s_x + 8, 0, NoHook{}, false, T(0), T(0));
            akkT = (T)s_d[1];
            akk = s_d[1];
            if (!isfinite(akkT)) { fail = ST_NONFINITE; break; }
        }
        PANEL_MARK(4);
        if (KEYS) {
            block_max2_u64(kl, ks, s_red2, red2_cnt);
            PANEL_MARK(11);
            // the two candidates' payloads and records from disjoint warps (threads 0..127 and
            // 128: lambda candidate; 256..383 and 384: sketch candidate), so that no thread
            // chains more than one of them before the barrier (d <= 128)
            if (kl != 0ull) {
                const int jc = (int)(kl & 0xFFFFull) - j_lo;
                if (tid < d) stcg(pay2 + (size_t)cta * ps + tid, Bs[(size_t)jc * ds + tid]);
                if (tid == 128) {
                    T *rp = reinterpret_cast<T *>(rec2 + 4 * (size_t)cta);
                    stcg(rp, c1[jc]);
                    stcg(rp + 1, dg[jc]);
                    red_max_u64(key_slot(keys, g2), kl);
                }
            }
            if (ks != 0ull) {
                const int jc = (int)(ks & 0xFFFFull) - j_lo;
                T *dst = spec_pay + (size_t)(par * G + cta) * ps;
                const int r = tid - 256;
                if (r >= 0 && r < d)
                    stcg(dst + r, deferred ? (T)(Bs[(size_t)jc * ds + r] - bP[r] * l1s[jc]) : Bs2[(size_t)jc * ds + r]);
                if (tid == 384) {
                    const T cv = c1[jc], l1 = cv * fk;
                    const T dnew = fma(-cv, l1, dg[jc]);
                    T *rp = reinterpret_cast<T *>(spec_rec + (size_t)(par * G + cta) * 4);
                    stcg(rp, dnew);
                    stcg(rp + 1, l1);
                    red_max_u64(key_slot(spec_keys, g2), ks);
                }
            }
        } else {
            CandT<T> c{T(-1), INT_MAX, -1};
            for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
                if (!alive[jl] || j_lo + jl == P) continue;
                T v = fabs(c1[jl]);
                if (better(v, lp[jl], c.v, c.lpos)) c = CandT<T>{v, lp[jl], j_lo + jl};
            }
            c = block_argmax(c, s_red);
            if (c.phys >= 0) {
                const int jc = c.phys - j_lo;
                for (int r = tid; r < d; r += PANEL_THREADS) stcg(pay2 + (size_t)cta * ps + r, Bs[(size_t)jc * ds + r]);
            }
            if (tid == 0) {
                s_i[9] = 0;
                const double cv = c.phys >= 0 ? (double)c1[c.phys - j_lo] : 0.0;
                const double dgc = c.phys >= 0 ? (double)dg[c.phys - j_lo] : 0.0;
                slot_write(rec2, cta, (double)c.v, cv, dgc, c.lpos, c.phys);
            }
        }
        PANEL_MARK(5);
        T tmaxLs = T(0);   // max |L(:, i)| of the speculative elimination
        if (KEYS) {
            grid_arrive(w.bar);
            if (spec) {
                // the case-(1) elimination of this step, speculatively, while thread 0 waits at the
                // barrier: W(:, i), the shadow diagonal dg2 and L(:, i).  A failed speculation
                // keeps dg, and the case (2)/(3) elimination rewrites W(:, i) and L(:, i) of every
                // live row (nothing reads them before that).
                for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
                    if (!alive[jl]) continue;
                    const int j = j_lo + jl;
                    T *wrow = Ws + (size_t)jl * ws;
                    T *lrow = w.Lg + (size_t)j * bw;
                    if (j == P) {
                        wrow[i] = T(0);
                        stcg(lrow + i, T(0));
                        continue;
                    }
                    const T cv = c1[jl];
                    const T l1 = cv * fk;
                    wrow[i] = cv;
                    dg2[jl] = fma(-cv, l1, dg[jl]);
                    stcg(lrow + i, l1);
                    tmaxLs = fmax(tmaxLs, fabs(l1));
                }
            }
            if (!grid_wait(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
        } else {
            if (!grid_barrier(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
        }
        PANEL_MARK(6);
        if (KEYS) {
            if (tid == 0) {
                const unsigned long long key = ld_key(key_slot(keys, g2));
                const unsigned long long key3 = spec ? ld_key(key_slot(spec_keys, g2)) : 0ull;
                if (cta == 0) *key_slot(keys, g2 + KEY_RING / 2) = 0ull;
                int R = -1, LR = -1;
                T lam = T(0);
                if (key != 0ull) {
                    R = (int)(key & 0xFFFFull);
                    LR = 0xFFFF - (int)((key >> 16) & 0xFFFFull);
                    lam = (T)__uint_as_float((unsigned)(key >> 32));
                }
                s_i[4] = R; s_i[5] = LR; s_i[6] = R >= 0 ? (R - k0) / chunk : 0;
                s_x[2] = lam;
                // SBKP test on the FP32 values, in FP32
                int kase;
                if (!isfinite(lam)) kase = -1;
                else if (lam == T(0)) kase = 0;
                else if (fabs(akkT) >= (T)alpha * lam) kase = 1;
                else kase = CASE_PENDING;
                if (kase == CASE_PENDING) {
                    s_i[7] = CASE_PENDING;
                } else {
                    // cases (0)/(1): the 1x1 pivot a_kk and its reciprocal, no FP64 arithmetic
                    s_i[7] = kase;
                    s_t[0] = s_t[1] = s_t[2] = T(0);
                    s_t[3] = T(1); s_t[4] = T(1);
                    s_t[5] = akkT;
                    s_t[6] = kase == 1 ? s_t[7] : T(0);
                    s_i[8] = akkT != T(0);
                }
                s_i[9] = 0;
                if (spec_keys && cta == 0) *key_slot(spec_keys, g2 + KEY_RING / 2) = 0ull;
                if (spec) {
                    if ((kase == 0 || kase == 1) && key3 != 0ull) {
                        s_i[9] = 1;   // commit the speculation
                        s_i[10] = (int)(key3 & 0xFFFFull);
                        s_i[11] = 0xFFFF - (int)((key3 >> 16) & 0xFFFFull);
                        s_i[12] = (s_i[10] - k0) / chunk;
                        s_x[6] = (T)__uint_as_float((unsigned)(key3 >> 32));
                    }
                }
            }
        } else if (warp == 0) {
            SlotWin b = slot_reduce(rec2, G);
            if (lane == 0) {
                const int R = b.phys;
                const double lam = R >= 0 ? b.v : 0.0, ark = R >= 0 ? b.a1 : 0.0, arr = R >= 0 ? b.a2 : 0.0;
                s_i[4] = R; s_i[5] = R >= 0 ? b.lpos : -1; s_i[6] = b.cta;
                s_d[2] = lam;
                int kase;
                if (!isfinite(lam) || !isfinite(ark) || !isfinite(arr)) kase = -1;
                else if (lam == 0.0) kase = 0;
                else if (fabs(akk) >= alpha * lam) kase = 1;
                else kase = fabs(arr) >= alpha * lam ? 2 : 3;
                sbkp_scalars<T>(kase, akk, lam, ark, arr, alpha, s_i, s_d, s_t, akk != 0.0 ? (T)(1.0 / akk) : T(0));
            }
        }
        __syncthreads();
        const int R = s_i[4], LR = s_i[5], gR = s_i[6];
        int kase = s_i[7];
        if (kase < 0) { fail = ST_NONFINITE; break; }
        if (s_i[9]) {
            PANEL_MARK(7);
            // case (0)/(1) confirmed: the speculative sketch update and elimination stand.  Issue
            // the loads of the next step (its pivot's column of A, sketch column, multipliers and
            // a_kk, the last multiplier coming with the speculation record), then adopt the
            // shadow sketch, norms and diagonal while they are in flight.
            const int P2 = s_i[10], LP2 = s_i[11], gc2 = s_i[12];
            preA0 = a_quad<T>(A, lda, j_lo, cnt, alive, P2, 0, P);
            preA1 = a_quad<T>(A, lda, j_lo, cnt, alive, P2, 1, P);
            const T pb = tid < d ? ldcg(spec_pay + (size_t)(par * G + gc2) * ps + tid) : T(0);
            const T pl = tid < i ? ldcg(w.Lg + (size_t)P2 * bw + tid) : T(0);
            T prec_d = T(0), prec_l = T(0);   // the next pivot's a_kk and L(P2, k), from its record
            if (tid == 0) {
                const T *rp = reinterpret_cast<const T *>(spec_rec + (size_t)(par * G + gc2) * 4);
                prec_d = ldcg(rp);
                prec_l = ldcg(rp + 1);
            }
            tmaxL = fmax(tmaxL, tmaxLs);
            PANEL_MARK(12);
            __syncthreads();
            PANEL_MARK(13);
            for (int jl = tid; jl < cnt; jl += PANEL_THREADS)
                if (j_lo + jl == P) alive[jl] = 0;
            if (deferred) {
                // the sketch update stays pending (bPd, l1s) until the next pass
                T *t = nrm; nrm = nrm2; nrm2 = t; t = dg; dg = dg2; dg2 = t;
                pend = true;
            } else {
                T *t = Bs; Bs = Bs2; Bs2 = t; t = nrm; nrm = nrm2; nrm2 = t; t = dg; dg = dg2; dg2 = t;
            }
            if (tid == 0) {
                ckind[i] = (kase == 0 || !s_i[8]) ? 0 : 1;
                cs0[i] = s_t[6];
                if (cta == 0) {
                    w.Dd[k] = (double)akkT; w.Ds[k] = 0.0;
                    maxDf = fmax(maxDf, fabs(akkT));
                    if (!s_i[8] && info == 0) info = k + 1;
                    minnorm2f = fminf((float)minnorm2f, (float)s_x[6]);
                }
                // the next step: pivot P2 to position k + 1
                const int kn = k + 1;
                const int Q = win[kn - k0];
                if (LP2 - k0 < wsz) win[LP2 - k0] = Q;
                win[kn - k0] = P2;
                if (P2 >= j_lo && P2 < j_lo + cnt) lp[P2 - j_lo] = kn;
                if (Q != P2 && Q >= j_lo && Q < j_lo + cnt) lp[Q - j_lo] = LP2;
                s_i[1] = P2; s_i[2] = LP2; s_i[3] = gc2;
                s_x[0] = s_x[6];
                s_x[8] = prec_d;            // a_kk of P2 after this step
                lP[i] = prec_l;             // L(P2, k)
            }
            if (tid < d) {
                if (deferred) bPd[tid] = bP[tid];   // the committed pivot's sketch column
                bP[tid] = pb;
            }
            if (tid < i) lP[tid] = pl;
            have_next = true;
            ++run1;
            PANEL_MARK(14);
            k += 1;
            i += 1;
            __syncthreads();
            continue;
        }
        have_next = false;
        run1 = kase <= 1 ? run1 + 1 : 0;
        PANEL_MARK(7);
        if (kase >= 2) {
            // column r of the Schur complement; in FP32 its record (a_rk, a_rr) arrives with the
            // column loads and thread 0 settles case 2 versus 3 right after them
            auto hook = [&]() {
                if (KEYS)
                    sbkp_scalars<T>(CASE_PENDING, (double)akkT, (double)s_x[2], (double)s_x[10], (double)s_x[11], alpha,
                                    s_i, s_d, s_t, s_t[7]);
            };
            schur_column<T>(A, lda, j_lo, cnt, R, i, ws, Ws, pay2 + (size_t)gR * ps, bR, w.Lg + (size_t)R * bw, lR, d,
                            alive, c2, reinterpret_cast<const T *>(rec2 + 4 * (size_t)gR), s_x + 10, KEYS ? 2 : 0, hook);
            kase = s_i[7];
            if (kase < 0) { fail = ST_NONFINITE; break; }
            if (tid == 0) {
                if (kase == 2) {
                    // interchange k <-> LR: R to position k, P to LR
                    int Q2 = win[k - k0];
                    if (LR - k0 < wsz) win[LR - k0] = Q2;
                    win[k - k0] = R;
                    if (R >= j_lo && R < j_lo + cnt) lp[R - j_lo] = k;
                    if (Q2 >= j_lo && Q2 < j_lo + cnt) lp[Q2 - j_lo] = LR;
                } else if (LR != k + 1) {
                    // interchange k+1 <-> LR: R to position k+1
                    int Q2 = win[k + 1 - k0];
                    if (LR - k0 < wsz) win[LR - k0] = Q2;
                    win[k + 1 - k0] = R;
                    if (R >= j_lo && R < j_lo + cnt) lp[R - j_lo] = k + 1;
                    if (Q2 >= j_lo && Q2 < j_lo + cnt) lp[Q2 - j_lo] = LR;
                }
            }
        }
        // ---------------- (4) multipliers, W, diagonal, sketch update ----------------
        PANEL_MARK(8);
        const int s = kase == 3 ? 2 : 1;
        const int piv1 = kase == 2 ? R : P;
        const int piv2 = kase == 3 ? R : -1;
        const double ark = s_d[3], arr = s_d[4], dpiv = s_d[5];
        const bool nonzero_piv = s_i[8] != 0;
        const T t_aa = s_t[0], t_cc = s_t[1], t_tinv = s_t[2], t_ark = s_t[3], t_rark = s_t[4];
        const T t_dpiv = s_t[5], t_rdpiv = s_t[6];
        const T *b1 = kase == 2 ? bR : bP;
        // four threads per owned row: multipliers (each of the four computes them), then the
        // row's sketch column with every fourth entry per thread
        const int sub = tid & 3;
        for (int jl0 = 0; jl0 < cnt; jl0 += PANEL_THREADS / 4) {
            const int jl = jl0 + (tid >> 2);
            bool live = jl < cnt && alive[jl];
            T sacc = T(0);
            if (live) {
                const int j = j_lo + jl;
                T *wrow = Ws + (size_t)jl * ws;
                T *lrow = w.Lg + (size_t)j * bw;
                if (j == piv1 || j == piv2) {
                    if (sub == 0) {
                        wrow[i] = T(0);
                        stcg(lrow + i, T(0));
                        if (s == 2) { wrow[i + 1] = T(0); stcg(lrow + i + 1, T(0)); }
                    }
                    live = false;
                } else {
                    T l1 = T(0), l2 = T(0);
                    if (kase <= 1) {
                        const T cv = c1[jl];
                        if (nonzero_piv) l1 = std::is_same<T, double>::value ? cv / t_dpiv : cv * t_rdpiv;
                        if (sub == 0) { wrow[i] = cv; dg[jl] = fma(-cv, l1, dg[jl]); }
                    } else if (kase == 2) {
                        const T cv = c2[jl];
                        l1 = std::is_same<T, double>::value ? cv / t_dpiv : cv * t_rdpiv;
                        if (sub == 0) { wrow[i] = cv; dg[jl] = fma(-cv, l1, dg[jl]); }
                    } else {
                        const T v1 = c1[jl], v2 = c2[jl];
                        const T x1 = std::is_same<T, double>::value ? v1 / t_ark : v1 * t_rark;
                        const T x2 = std::is_same<T, double>::value ? v2 / t_ark : v2 * t_rark;
                        l1 = t_tinv * (t_cc * x1 - x2);
                        l2 = t_tinv * (t_aa * x2 - x1);
                        if (sub == 0) { wrow[i] = v1; wrow[i + 1] = v2; dg[jl] = dg[jl] - v1 * l1 - v2 * l2; }
                    }
                    if (sub == 1) {
                        stcg(lrow + i, l1);
                        if (s == 2) stcg(lrow + i + 1, l2);
                    }
                    tmaxL = fmax(tmaxL, fmax(fabs(l1), fabs(l2)));
                    T *col = Bs + (size_t)jl * ds;
                    if (w.qb) {
                        // q = b: the sketch is updated once per block, after the panel
                    } else {
                        // rows sub, sub+4, ...: five at a time, loads of a chunk before its stores
                        for (int r0 = sub; r0 < d; r0 += 20) {
                            T v[5], p1[5], p2[5];
#pragma unroll
                            for (int q = 0; q < 5; ++q) {
                                const int r = r0 + 4 * q;
                                v[q] = r < d ? col[r] : T(0);
                                p1[q] = r < d ? b1[r] : T(0);
                                p2[q] = (r < d && s == 2) ? bR[r] : T(0);
                            }
#pragma unroll
                            for (int q = 0; q < 5; ++q) {
                                const int r = r0 + 4 * q;
                                const T x = v[q] - p1[q] * l1 - p2[q] * l2;
                                if (r < d) col[r] = x;
                                sacc = fma(x, x, sacc);
                            }
                        }
                    }
                }
            }
            sacc += __shfl_xor_sync(FULL, sacc, 1);
            sacc += __shfl_xor_sync(FULL, sacc, 2);
            if (live && sub == 0) nrm[jl] = sacc;
        }
        __syncthreads();
        // pivots leave the active set only after every quad has read alive[]
        for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
            const int j = j_lo + jl;
            if (alive[jl] && (j == piv1 || j == piv2)) alive[jl] = 0;
        }
        PANEL_MARK(9);
        if (tid == 0) {
            // the D scalars of this step, so that any row's L entries can be rebuilt from W
            if (kase == 3) {
                ckind[i] = 3; ckind[i + 1] = 4;
                cs0[i] = t_aa; cs1[i] = t_cc; cs2[i] = t_tinv;
                cs3[i] = std::is_same<T, double>::value ? t_ark : t_rark;
            } else {
                ckind[i] = (kase == 0 || !nonzero_piv) ? 0 : 1;
                cs0[i] = std::is_same<T, double>::value ? t_dpiv : t_rdpiv;
            }
        }
        if (cta == 0 && tid == 0) {
            const double akk_d = KEYS ? (double)akkT : akk;
            if (kase == 3) {
                w.Dd[k] = akk_d; w.Ds[k] = ark; w.Dd[k + 1] = arr; w.Ds[k + 1] = 0.0;
                maxD = fmax(maxD, fmax(fabs(akk_d), fmax(fabs(ark), fabs(arr))));
                ++n2;
            } else {
                const double dp = KEYS ? (double)s_t[5] : dpiv;
                w.Dd[k] = dp; w.Ds[k] = 0.0;
                maxD = fmax(maxD, fabs(dp));
                if (!nonzero_piv && info == 0) info = k + 1;
            }
        }
        k += s;
        i += s;
        __syncthreads();
    }
#undef PANEL_MARK

    // ---------------- epilogue: publish the panel in logical order ----------------
    __syncthreads();
    if (pend) {
        // deferred: a confirmed speculative update that no later pass applied (the loop ended)
        for (int e = tid; e < cnt * d; e += PANEL_THREADS) {
            const int jl = e / d, r = e - jl * d;
            if (alive[jl]) Bs[(size_t)jl * ds + r] = Bs[(size_t)jl * ds + r] - bPd[r] * l1s[jl];
        }
        __syncthreads();
    }
    T amw = T(0), aml = T(0);   // max |W| and |L| over the rows left for the trailing update
    for (int e = tid; e < cnt * i; e += PANEL_THREADS) {
        int t = e / cnt, jl = e - t * cnt;
        const T *wrow = Ws + (size_t)jl * ws;
        const T lv = l_entry<T>(wrow, t, ckind, cs0, cs1, cs2, cs3);
        if (alive[jl]) {
            w.Wbuf[(size_t)lp[jl] + (size_t)t * n] = wrow[t];
            amw = fmax(amw, fabs(wrow[t]));
            aml = fmax(aml, fabs(lv));
        }
        w.Lc[(size_t)lp[jl] + (size_t)t * n] = lv;
    }
    for (int e = tid; e < cnt * d; e += PANEL_THREADS) {
        int jl = e / d, r = e - jl * d;
        if (alive[jl] || w.qb) w.B[(size_t)r + (size_t)lp[jl] * d] = Bs[(size_t)jl * ds + r];
    }
    // the moved rows, appended with one atomic per warp (the CTAs that own the panel's
    // positions move nearly every row), with their position marks and saved permutation entries
    // for the interchange kernels (phi: second half of the moved buffer)
    int *const phi = w.moved + n;
    for (int base = 0; base < cnt; base += PANEL_THREADS) {
        const int jl = base + tid, j = j_lo + jl;
        bool mv = false;
        if (jl < cnt) {
            w.lpos[j] = lp[jl];
            mv = lp[jl] != j;
        }
        const unsigned bal = __ballot_sync(FULL, mv);
        if (bal != 0u) {
            int first = 0;
            if (lane == 0) first = atomicAdd(&w.st->n_moved, __popc(bal));
            first = __shfl_sync(FULL, first, 0);
            if (mv) {
                const int idx = first + __popc(bal & ((1u << lane) - 1u));
                if (idx < w.maxmoved) {
                    w.moved[idx] = j;
                    phi[lp[jl]] = j;
                    w.tmpP[idx] = w.perm[j];
                } else {
                    atomicOr(w.status, ST_INTERNAL);
                }
            }
        }
    }
    // per-CTA statistics
    {
        double v = (double)tmaxL;
        for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, off));
        if (lane == 0 && v > 0.0) atomic_max_nonneg(&w.st->maxL_bits, v);
    }
    // panel maxima of |W| and |L21| over the trailing rows (scales of the FP16 split update):
    // per block, then one atomic pair per CTA
    {
        __shared__ T s_am[2][PANEL_WARPS];
        for (int off = 16; off > 0; off >>= 1) {
            amw = fmax(amw, __shfl_xor_sync(FULL, amw, off));
            aml = fmax(aml, __shfl_xor_sync(FULL, aml, off));
        }
        if (lane == 0) { s_am[0][warp] = amw; s_am[1][warp] = aml; }
        __syncthreads();
        if (tid == 0) {
            for (int q = 1; q < PANEL_WARPS; ++q) { amw = fmax(amw, s_am[0][q]); aml = fmax(aml, s_am[1][q]); }
            if (amw > T(0)) atomic_max_nonneg(&w.st->tcW_bits, (double)amw);
            if (aml > T(0)) atomic_max_nonneg(&w.st->tcL_bits, (double)aml);
        }
    }
    if (tid == 0 && cta == 0) {
        if (KEYS) {
            if (beta2f > T(0)) {
                beta2 = (double)beta2f;
                w.st->beta2 = beta2;
            }
            minnorm2 = fmin(minnorm2, (double)minnorm2f);
            maxD = fmax(maxD, (double)maxDf);
        }
        if (fail) {
            atomicOr(w.status, fail);
            w.st->next = n;
        } else {
            w.st->next = k;
        }
        w.st->k0 = k0;
        w.st->kend = k;
        w.st->n2x2 += n2;
        w.st->guard_req = gstop ? (ldcg(&w.st->nresk) + 1 < w.guard_r ? 1 : 2) : 0;
        if (gstop) w.st->guard_k = k;
        if (info && w.st->info == 0) w.st->info = info;
        if (beta2 > 0.0 && minnorm2 < INFINITY) {
            const double ratio = sqrt(minnorm2 / beta2);
            if (ratio < w.st->min_ratio) w.st->min_ratio = ratio;
        }
        atomic_max_nonneg(&w.st->maxD_bits, maxD);
    }
}

// Largest dynamic shared memory the panel kernel may request (opt-in limit minus its static
// shared memory); the attribute is set once per instantiation.
template <typename T, bool DEF>
static size_t panel_dyn_limit() {
    static size_t limit = 0;
    if (limit == 0) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, panel_kernel<T, DEF>) != cudaSuccess) return 0;
        size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        if (cudaFuncSetAttribute(panel_kernel<T, DEF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) != cudaSuccess)
            return 0;
        limit = lim;
    }
    return limit;
}

template <typename T>
cudaError_t launch_panel(const FactorWork<T> &w, cudaStream_t s) {
    size_t smem = panel_smem_bytes<T>(w.d, w.bw, w.chunk_cap, w.spec);
    FactorWork<T> arg = w;
    void *args[] = {&arg};
    if constexpr (std::is_same<T, float>::value) {
        if (w.spec == 2) {
            if (smem > panel_dyn_limit<T, true>()) return cudaErrorInvalidValue;
            count_launches(1);
            return cudaLaunchCooperativeKernel((const void *)panel_kernel<T, true>, dim3(w.grid), dim3(PANEL_THREADS), args,
                                               smem, s);
        }
    }
    if (smem > panel_dyn_limit<T, false>()) return cudaErrorInvalidValue;
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)panel_kernel<T, false>, dim3(w.grid), dim3(PANEL_THREADS), args, smem, s);
}

// Largest cooperative grid for the given per-CTA workspace (0 if it does not fit).
template <typename T>
int panel_max_grid(int d, int bw, int chunk_cap, int spec) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t smem = panel_smem_bytes<T>(d, bw, chunk_cap, spec);
    if constexpr (std::is_same<T, float>::value) {
        if (spec == 2) {
            if (smem > panel_dyn_limit<T, true>()) return 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, panel_kernel<T, true>, PANEL_THREADS, smem) != cudaSuccess)
                return 0;
            return per * sms;
        }
    }
    if (smem > panel_dyn_limit<T, false>()) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, panel_kernel<T, false>, PANEL_THREADS, smem) != cudaSuccess)
        return 0;
    return per * sms;
}

// The panel's grid-wide exchange without its arithmetic, for a latency floor of the pivot
// step: per round every CTA's thread 0 adds a packed key to a ring slot by red.max, the CTA
// arrives at the grid barrier and waits, thread 0 reads the slot back, and CTA 0 clears the slot
// half a ring ahead (as the FP32 panel does once per pivot step in its speculative path).
__global__ void __launch_bounds__(PANEL_THREADS, 1) exchange_probe_kernel(unsigned *bar, unsigned long long *keys,
                                                                          int *status, int rounds) {
    __shared__ unsigned s_base;
    const unsigned G = gridDim.x;
    if (threadIdx.x == 0) s_base = barrier_base(bar, G);
    __syncthreads();
    const unsigned base = s_base;
    unsigned long long acc = 0ull;
    for (int r = 0; r < rounds; ++r) {
        if (threadIdx.x == 0)
            red_max_u64(key_slot(keys, (unsigned)r), make_key((float)(blockIdx.x + 1), r & 0xFFFF, (int)blockIdx.x));
        if (!grid_barrier(bar, base + (unsigned)(r + 1) * G, status)) return;
        if (threadIdx.x == 0) {
            acc += ld_key(key_slot(keys, (unsigned)r)) & 0xFFFFull;   // the winning CTA of the round
            if (blockIdx.x == 0) *key_slot(keys, (unsigned)(r + KEY_RING / 2)) = 0ull;
        }
        __syncthreads();
    }
    // every round is won by the last CTA: a wrong exchange shows up in the status word
    if (threadIdx.x == 0 && acc != (unsigned long long)rounds * (G - 1)) atomicOr(status, ST_INTERNAL);
}

// Failure path of the bounded waits: every CTA arrives once at a grid barrier whose target is
// one arrival more than the launch has CTAs, so no wait can complete; each CTA gives up after
// limit_ns, sets ST_TIMEOUT and returns.  CTA 0 records how long its wait lasted.
__global__ void __launch_bounds__(PANEL_THREADS, 1) wait_expiry_kernel(unsigned *bar, int *status,
                                                                        unsigned long long limit_ns,
                                                                        unsigned long long *elapsed_ns) {
    __shared__ unsigned s_base;
    const unsigned G = gridDim.x;
    if (threadIdx.x == 0) s_base = barrier_base(bar, G);
    __syncthreads();
    const unsigned long long t0 = global_ns();
    const bool ok = grid_barrier(bar, s_base + G + 1u, status, limit_ns);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *elapsed_ns = global_ns() - t0;
        if (ok) atomicOr(status, ST_INTERNAL);   // a barrier nobody can complete did complete
    }
}

cudaError_t launch_wait_expiry(unsigned *bar, int *status, int grid, unsigned long long limit_ns,
                               unsigned long long *elapsed_ns, cudaStream_t s) {
    void *args[] = {&bar, &status, &limit_ns, &elapsed_ns};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)wait_expiry_kernel, dim3(grid), dim3(PANEL_THREADS), args, 0, s);
}

int exchange_probe_grid() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, exchange_probe_kernel, PANEL_THREADS, 0) != cudaSuccess)
        return 0;
    return per * sms;
}

cudaError_t launch_exchange_probe(unsigned *bar, unsigned long long *keys, int *status, int grid, int rounds,
                                  cudaStream_t s) {
    void *args[] = {&bar, &keys, &status, &rounds};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)exchange_probe_kernel, dim3(grid), dim3(PANEL_THREADS), args, 0, s);
}

template size_t panel_smem_bytes<double>(int, int, int, int);
template size_t panel_smem_bytes<float>(int, int, int, int);
template cudaError_t launch_panel<double>(const FactorWork<double> &, cudaStream_t);
template cudaError_t launch_panel<float>(const FactorWork<float> &, cudaStream_t);
template int panel_max_grid<double>(int, int, int, int);
template int panel_max_grid<float>(int, int, int, int);

}  // namespace rcpk
