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
// interchange kernels (interchange.cu).
//
// Per pivot step (Section 3, Figure SBKP, Eq. "Update matrix B"):
//   (1) argmax of ||B(:, j)||^2 over the remaining indices (ties: smallest position)  -> P
//       grid barrier #1 (each CTA publishes its best candidate and that candidate's B column)
//   (2) the interchange k <-> position(P); column P of the Schur complement,
//       c_j = A(j, P) - sum_t W(j, t) L(P, t) (a GEMV over the panel built so far);
//       lambda = max_{j != P} |c_j| at r (ties: smallest position)
//       grid barrier #2 (best candidate, its c value, its current diagonal, its B column)
//   (3) SBKP case (0)-(3) with alpha; for cases (2)/(3) column r of the Schur complement
//   (4) multipliers (1x1: c / a_kk; 2x2: [c_j c'_j] D_k^{-1} in FP64), W = L D, the
//       Schur diagonal update, and the rank-s sketch update fused with the next norms.
// So one pivot step (1x1 or 2x2) costs two grid-wide barriers.
#include <climits>

#include "kernels.h"

namespace rcpk {

constexpr int PANEL_THREADS = 512;
constexpr int PANEL_WARPS = PANEL_THREADS / 32;
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
size_t panel_smem_bytes(int d, int bw, int chunk_cap) {
    size_t s = 0;
    s += (size_t)chunk_cap * sizeof(double);           // nrm
    s += (size_t)chunk_cap * d * sizeof(T);            // Bs
    s += (size_t)chunk_cap * bw * sizeof(T);           // Ws
    s += (size_t)chunk_cap * 5 * sizeof(T);            // dg, c1, c2, l1s, l2s
    s += (size_t)2 * d * sizeof(T);                    // bP, bR
    s += (size_t)2 * bw * sizeof(T);                   // lP, lR
    s += (size_t)chunk_cap * 2 * sizeof(int);          // lp, alive
    s += (size_t)(bw + 3) * sizeof(int);               // window
    return s + 64;
}

struct Cand {
    double v;
    int lpos;
    int phys;
};

__device__ __forceinline__ bool better(double v1, int l1, double v2, int l2) {
    return v1 > v2 || (v1 == v2 && l1 < l2);
}

__device__ __forceinline__ Cand warp_argmax(Cand c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        double v = __shfl_down_sync(FULL, c.v, off);
        int l = __shfl_down_sync(FULL, c.lpos, off);
        int p = __shfl_down_sync(FULL, c.phys, off);
        if (better(v, l, c.v, c.lpos)) { c.v = v; c.lpos = l; c.phys = p; }
    }
    return c;
}

// Block-wide argmax; the result is returned to every thread.
__device__ __forceinline__ Cand block_argmax(Cand c, Cand *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    c = warp_argmax(c);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    if (warp == 0) {
        Cand x = lane < PANEL_WARPS ? red[lane] : Cand{-1.0, INT_MAX, -1};
        x = warp_argmax(x);
        if (lane == 0) red[PANEL_WARPS] = x;
    }
    __syncthreads();
    Cand r = red[PANEL_WARPS];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double warp_sum(double s) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
    return s;
}

template <typename T>
__device__ __forceinline__ T a_sym(const T *__restrict__ A, int lda, int i, int j) {
    return i >= j ? A[(size_t)i + (size_t)j * lda] : A[(size_t)j + (size_t)i * lda];
}

// Reads G slots (value, position, index) and returns the winning CTA (warp 0 only).
__device__ __forceinline__ int slot_winner(const double *sv, int vstride, const int *si, int G) {
    const int lane = threadIdx.x & 31;
    Cand c{-1.0, INT_MAX, lane};
    for (int g = lane; g < G; g += 32) {
        double v = ldcg(sv + (size_t)g * vstride);
        int l = ldcg(si + 2 * (size_t)g);
        if (better(v, l, c.v, c.lpos)) { c.v = v; c.lpos = l; c.phys = g; }
    }
    c = warp_argmax(c);
    return __shfl_sync(FULL, c.phys, 0);
}

// c[jl] = A(j, X) - sum_{t < i} Ws[jl][t] lX[t] for the alive owned rows.
template <typename T>
__device__ void schur_column(const T *__restrict__ A, int lda, int j_lo, int cnt, int X, int i, int bw,
                             const T *Ws, const T *lX, const int *alive, T *c) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // issue the column loads first (at most two rows per thread)
    T a0 = T(0), a1 = T(0);
    const int r0 = threadIdx.x, r1 = threadIdx.x + PANEL_THREADS;
    if (r0 < cnt && alive[r0]) a0 = a_sym(A, lda, j_lo + r0, X);
    if (r1 < cnt && alive[r1]) a1 = a_sym(A, lda, j_lo + r1, X);
    if (i > 0) {
        for (int jl = warp; jl < cnt; jl += PANEL_WARPS) {
            if (!alive[jl]) continue;
            double s = 0.0;
            for (int t = lane; t < i; t += 32) s += (double)(Ws[(size_t)jl * bw + t] * lX[t]);
            s = warp_sum(s);
            if (lane == 0) c[jl] = (T)s;
        }
    } else {
        for (int jl = threadIdx.x; jl < cnt; jl += PANEL_THREADS) c[jl] = T(0);
    }
    __syncthreads();
    if (r0 < cnt) c[r0] = alive[r0] ? (T)(a0 - c[r0]) : T(0);
    if (r1 < cnt) c[r1] = alive[r1] ? (T)(a1 - c[r1]) : T(0);
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS, 1) panel_kernel(FactorWork<T> w) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Cand s_red[PANEL_WARPS + 1];
    __shared__ int s_i[16];
    __shared__ double s_d[16];

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

    double *nrm = reinterpret_cast<double *>(smem);
    T *Bs = reinterpret_cast<T *>(nrm + cap);
    T *Ws = Bs + (size_t)cap * d;
    T *dg = Ws + (size_t)cap * bw;
    T *c1 = dg + cap;
    T *c2 = c1 + cap;
    T *l1s = c2 + cap;
    T *l2s = l1s + cap;
    T *bP = l2s + cap;
    T *bR = bP + d;
    T *lP = bR + d;
    T *lR = lP + bw;
    int *lp = reinterpret_cast<int *>(lR + bw);
    int *alive = lp + cap;
    int *win = alive + cap;           // positions k0 .. k0 + bw + 2
    const int wsz = bw + 3;

    const T *__restrict__ A = w.A;
    // ---- load the owned state ----
    for (int e = tid; e < cnt * d; e += PANEL_THREADS) {
        int jl = e / d, r = e - jl * d;
        Bs[e] = w.B[(size_t)r + (size_t)(j_lo + jl) * d];
    }
    for (int e = tid; e < cnt * bw; e += PANEL_THREADS) Ws[e] = T(0);
    for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
        int j = j_lo + jl;
        dg[jl] = A[(size_t)j + (size_t)j * lda];
        lp[jl] = j;
        alive[jl] = 1;
    }
    for (int x = tid; x < wsz; x += PANEL_THREADS) win[x] = k0 + x;
    if (tid == 0) {
        s_i[0] = (int)barrier_base(w.bar, (unsigned)G);
        if (cta == 0) w.st->n_moved = 0;
    }
    __syncthreads();
    // initial column norms
    for (int jl = warp; jl < cnt; jl += PANEL_WARPS) {
        double s = 0.0;
        for (int r = lane; r < d; r += 32) { double b = (double)Bs[(size_t)jl * d + r]; s += b * b; }
        s = warp_sum(s);
        if (lane == 0) nrm[jl] = s;
    }
    const unsigned base = (unsigned)s_i[0];
    unsigned nbar = 0;
    int k = k0, i = 0, n2 = 0;
    double maxL = 0.0, maxD = 0.0, minratio = 2.0;
    int info = 0, fail = 0;
    const double alpha = w.alpha;
    T *pay1 = w.pay, *pay2 = w.pay + (size_t)G * d;
    __syncthreads();

    while (i < w.bmax && k < n) {
        // ---------------- (1) sketch column-norm argmax ----------------
        Cand c{-1.0, INT_MAX, -1};
        for (int jl = tid; jl < cnt; jl += PANEL_THREADS)
            if (alive[jl] && better(nrm[jl], lp[jl], c.v, c.lpos)) c = Cand{nrm[jl], lp[jl], j_lo + jl};
        c = block_argmax(c, s_red);
        if (c.phys >= 0)
            for (int r = tid; r < d; r += PANEL_THREADS) stcg(pay1 + (size_t)cta * d + r, Bs[(size_t)(c.phys - j_lo) * d + r]);
        if (tid == 0) {
            stcg(w.s1v + 2 * (size_t)cta, c.v);
            stcg(w.s1v + 2 * (size_t)cta + 1, c.phys >= 0 ? (double)dg[c.phys - j_lo] : 0.0);
            stcg(w.s1i + 2 * (size_t)cta, c.lpos);
            stcg(w.s1i + 2 * (size_t)cta + 1, c.phys);
        }
        if (!grid_barrier(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
        if (warp == 0) {
            int g = slot_winner(w.s1v, 2, w.s1i, G);
            if (lane == 0) {
                s_i[1] = ldcg(w.s1i + 2 * (size_t)g + 1);   // P
                s_i[2] = ldcg(w.s1i + 2 * (size_t)g);       // position of P
                s_i[3] = g;
                s_d[0] = ldcg(w.s1v + 2 * (size_t)g);       // ||B(:, P)||^2
                s_d[1] = ldcg(w.s1v + 2 * (size_t)g + 1);   // a_kk
            }
        }
        __syncthreads();
        const int P = s_i[1], LP = s_i[2], gP = s_i[3];
        const double norm2 = s_d[0], akk = s_d[1];
        if (P < 0 || !isfinite(norm2) || !isfinite(akk)) { fail = ST_NONFINITE; break; }
        for (int r = tid; r < d; r += PANEL_THREADS) bP[r] = ldcg(pay1 + (size_t)gP * d + r);
        for (int t = tid; t < i; t += PANEL_THREADS) lP[t] = ldcg(w.Lp + (size_t)P * bw + t);
        if (tid == 0) {
            // interchange k <-> LP (positions); Q is the index now at position k
            int Q = win[k - k0];
            if (LP - k0 < wsz) win[LP - k0] = Q;
            win[k - k0] = P;
            if (P >= j_lo && P < j_lo + cnt) lp[P - j_lo] = k;
            if (Q != P && Q >= j_lo && Q < j_lo + cnt) lp[Q - j_lo] = LP;
            if (cta == 0) {
                if (k == 0) w.st->beta2 = norm2;
                double b2 = (k == 0) ? norm2 : ldcg(&w.st->beta2);
                if (b2 > 0.0) minratio = fmin(minratio, sqrt(norm2 / b2));
            }
        }
        __syncthreads();

        // ---------------- (2) column P of the Schur complement, lambda and r ----------------
        schur_column<T>(A, lda, j_lo, cnt, P, i, bw, Ws, lP, alive, c1);
        c = Cand{-1.0, INT_MAX, -1};
        for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
            if (!alive[jl] || j_lo + jl == P) continue;
            double v = fabs((double)c1[jl]);
            if (better(v, lp[jl], c.v, c.lpos)) c = Cand{v, lp[jl], j_lo + jl};
        }
        c = block_argmax(c, s_red);
        if (c.phys >= 0)
            for (int r = tid; r < d; r += PANEL_THREADS) stcg(pay2 + (size_t)cta * d + r, Bs[(size_t)(c.phys - j_lo) * d + r]);
        if (tid == 0) {
            stcg(w.s2v + 3 * (size_t)cta, c.v);
            stcg(w.s2v + 3 * (size_t)cta + 1, c.phys >= 0 ? (double)c1[c.phys - j_lo] : 0.0);
            stcg(w.s2v + 3 * (size_t)cta + 2, c.phys >= 0 ? (double)dg[c.phys - j_lo] : 0.0);
            stcg(w.s2i + 2 * (size_t)cta, c.lpos);
            stcg(w.s2i + 2 * (size_t)cta + 1, c.phys);
        }
        if (!grid_barrier(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
        if (warp == 0) {
            int g = slot_winner(w.s2v, 3, w.s2i, G);
            if (lane == 0) {
                s_i[4] = ldcg(w.s2i + 2 * (size_t)g + 1);   // R (or -1)
                s_i[5] = ldcg(w.s2i + 2 * (size_t)g);       // position of R
                s_i[6] = g;
                s_d[2] = ldcg(w.s2v + 3 * (size_t)g);       // lambda
                s_d[3] = ldcg(w.s2v + 3 * (size_t)g + 1);   // a_rk
                s_d[4] = ldcg(w.s2v + 3 * (size_t)g + 2);   // a_rr
            }
        }
        __syncthreads();
        const int R = s_i[4], LR = s_i[5], gR = s_i[6];
        const double lam = R >= 0 ? s_d[2] : 0.0, ark = s_d[3], arr = s_d[4];
        if (!isfinite(lam) || (R >= 0 && (!isfinite(ark) || !isfinite(arr)))) { fail = ST_NONFINITE; break; }

        // ---------------- (3) SBKP ----------------
        int kase;
        if (lam == 0.0) kase = 0;
        else if (fabs(akk) >= alpha * lam) kase = 1;
        else if (fabs(arr) >= alpha * lam) kase = 2;
        else kase = 3;
        const int s = kase == 3 ? 2 : 1;
        if (kase >= 2) {
            for (int r = tid; r < d; r += PANEL_THREADS) bR[r] = ldcg(pay2 + (size_t)gR * d + r);
            for (int t = tid; t < i; t += PANEL_THREADS) lR[t] = ldcg(w.Lp + (size_t)R * bw + t);
            __syncthreads();
            schur_column<T>(A, lda, j_lo, cnt, R, i, bw, Ws, lR, alive, c2);
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
        const int piv1 = kase == 2 ? R : P;
        const int piv2 = kase == 3 ? R : -1;
        // 2x2 inverse in FP64, scaled by the off-diagonal entry
        const double aa = kase == 3 ? akk / ark : 0.0, cc = kase == 3 ? arr / ark : 0.0;
        const double tinv = kase == 3 ? 1.0 / (aa * cc - 1.0) : 0.0;
        const double dpiv = kase == 2 ? arr : akk;
        for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
            if (!alive[jl]) continue;
            const int j = j_lo + jl;
            T *wrow = Ws + (size_t)jl * bw;
            T *lrow = w.Lp + (size_t)j * bw;
            if (j == piv1 || j == piv2) {
                wrow[i] = T(0);
                stcg(lrow + i, T(0));
                if (s == 2) { wrow[i + 1] = T(0); stcg(lrow + i + 1, T(0)); }
                alive[jl] = 0;
                continue;
            }
            double l1 = 0.0, l2 = 0.0;
            if (kase <= 1) {
                double cv = (double)c1[jl];
                l1 = dpiv != 0.0 ? cv / dpiv : 0.0;
                wrow[i] = c1[jl];
                dg[jl] = (T)((double)dg[jl] - cv * l1);
            } else if (kase == 2) {
                double cv = (double)c2[jl];
                l1 = cv / dpiv;
                wrow[i] = c2[jl];
                dg[jl] = (T)((double)dg[jl] - cv * l1);
            } else {
                double x1 = (double)c1[jl] / ark, x2 = (double)c2[jl] / ark;
                l1 = tinv * (cc * x1 - x2);
                l2 = tinv * (aa * x2 - x1);
                wrow[i] = c1[jl];
                wrow[i + 1] = c2[jl];
                dg[jl] = (T)((double)dg[jl] - (double)c1[jl] * l1 - (double)c2[jl] * l2);
            }
            T tl1 = (T)l1, tl2 = (T)l2;
            stcg(lrow + i, tl1);
            if (s == 2) stcg(lrow + i + 1, tl2);
            l1s[jl] = tl1;
            l2s[jl] = tl2;
            maxL = fmax(maxL, fmax(fabs(l1), fabs(l2)));
        }
        __syncthreads();
        // rank-s sketch update fused with the next column norms
        const T *b1 = kase == 2 ? bR : bP;
        for (int jl = warp; jl < cnt; jl += PANEL_WARPS) {
            if (!alive[jl]) continue;
            const T f1 = l1s[jl], f2 = l2s[jl];
            T *col = Bs + (size_t)jl * d;
            double sacc = 0.0;
            if (s == 2) {
                for (int r = lane; r < d; r += 32) {
                    T v = col[r] - b1[r] * f1 - bR[r] * f2;
                    col[r] = v;
                    sacc += (double)v * (double)v;
                }
            } else {
                for (int r = lane; r < d; r += 32) {
                    T v = col[r] - b1[r] * f1;
                    col[r] = v;
                    sacc += (double)v * (double)v;
                }
            }
            sacc = warp_sum(sacc);
            if (lane == 0) nrm[jl] = sacc;
        }
        if (cta == 0 && tid == 0) {
            if (kase == 3) {
                w.Dd[k] = akk; w.Ds[k] = ark; w.Dd[k + 1] = arr; w.Ds[k + 1] = 0.0;
                maxD = fmax(maxD, fmax(fabs(akk), fmax(fabs(ark), fabs(arr))));
                ++n2;
            } else {
                w.Dd[k] = dpiv; w.Ds[k] = 0.0;
                maxD = fmax(maxD, fabs(dpiv));
                if (dpiv == 0.0 && info == 0) info = k + 1;
            }
        }
        k += s;
        i += s;
        __syncthreads();
    }

    // ---------------- epilogue: publish the panel in logical order ----------------
    __syncthreads();
    for (int e = tid; e < cnt * i; e += PANEL_THREADS) {
        int t = e / cnt, jl = e - t * cnt;
        if (alive[jl]) w.Wbuf[(size_t)lp[jl] + (size_t)t * n] = Ws[(size_t)jl * bw + t];
    }
    for (int e = tid; e < cnt * d; e += PANEL_THREADS) {
        int jl = e / d, r = e - jl * d;
        if (alive[jl]) w.B[(size_t)r + (size_t)lp[jl] * d] = Bs[e];
    }
    for (int jl = tid; jl < cnt; jl += PANEL_THREADS) {
        int j = j_lo + jl;
        w.lpos[j] = lp[jl];
        if (lp[jl] != j) {
            int idx = atomicAdd(&w.st->n_moved, 1);
            if (idx < w.maxmoved) w.moved[idx] = j;
            else atomicOr(w.status, ST_INTERNAL);
        }
    }
    // per-CTA statistics
    {
        double v = maxL;
        for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, off));
        if (lane == 0 && v > 0.0) atomic_max_nonneg(&w.st->maxL_bits, v);
    }
    if (tid == 0 && cta == 0) {
        if (fail) {
            atomicOr(w.status, fail);
            w.st->next = n;
        } else {
            w.st->next = k;
        }
        w.st->k0 = k0;
        w.st->kend = k;
        w.st->n2x2 += n2;
        if (info && w.st->info == 0) w.st->info = info;
        if (minratio < w.st->min_ratio) w.st->min_ratio = minratio;
        atomic_max_nonneg(&w.st->maxD_bits, maxD);
    }
}

// Largest dynamic shared memory the panel kernel may request (opt-in limit minus its static
// shared memory); the attribute is set once per instantiation.
template <typename T>
static size_t panel_dyn_limit() {
    static size_t limit = 0;
    if (limit == 0) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, panel_kernel<T>) != cudaSuccess) return 0;
        size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        if (cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) != cudaSuccess)
            return 0;
        limit = lim;
    }
    return limit;
}

template <typename T>
cudaError_t launch_panel(const FactorWork<T> &w, cudaStream_t s) {
    size_t smem = panel_smem_bytes<T>(w.d, w.bw, w.chunk_cap);
    if (smem > panel_dyn_limit<T>()) return cudaErrorInvalidValue;
    FactorWork<T> arg = w;
    void *args[] = {&arg};
    return cudaLaunchCooperativeKernel((const void *)panel_kernel<T>, dim3(w.grid), dim3(PANEL_THREADS), args, smem, s);
}

// Largest cooperative grid for the given per-CTA workspace (0 if it does not fit).
template <typename T>
int panel_max_grid(int d, int bw, int chunk_cap) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t smem = panel_smem_bytes<T>(d, bw, chunk_cap);
    if (smem > panel_dyn_limit<T>()) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, panel_kernel<T>, PANEL_THREADS, smem) != cudaSuccess) return 0;
    return per * sms;
}

template size_t panel_smem_bytes<double>(int, int, int);
template size_t panel_smem_bytes<float>(int, int, int);
template cudaError_t launch_panel<double>(const FactorWork<double> &, cudaStream_t);
template cudaError_t launch_panel<float>(const FactorWork<float> &, cudaStream_t);
template int panel_max_grid<double>(int, int, int);
template int panel_max_grid<float>(int, int, int);

}  // namespace rcpk
