// interchange.cu -- applies one panel's symmetric interchanges to the stored arrays and
// performs the deferred trailing update of Algorithm 1 ("compute Schur complement"); also the
// start and end of a factorization, and the zero fill of the Schur complement where the
// Algorithm 2 safeguard stops.
//
// After a panel, position p >= k0 holds the block-start index phi(p); only a few indices
// moved (at most twice the panel width).  For each moved index j with new position
// p = lpos[j]:
//   perm[p]              <- perm[j]
//   A_sym(p, q), q >= kend <- A_sym(j, phi(q))         (only when p itself is >= kend)
// done as a gather into scratch followed by a scatter (two launches, so no read sees a
// half-written line).  Then the panel's multipliers go to A(:, k0:kend) in position order,
// and the trailing update A22 -= W L21^T runs on the lower triangle of A(kend:n, kend:n).
// The rows of the earlier L columns (L(p, 0:k0) <- L(j, 0:k0)) are not moved here: nothing
// reads them before the factorization ends, so the permutation after every panel is recorded
// and each panel's L columns are permuted once at the end (the deferred row interchanges of
// blocked LAPACK factorizations), with column-contiguous accesses instead of strided rows.
#include <algorithm>

#include "kernels.h"

namespace rcpk {

template <typename T>
__device__ __forceinline__ T a_sym_ld(const T *__restrict__ A, int lda, int i, int j) {
    return i >= j ? A[(size_t)i + (size_t)j * lda] : A[(size_t)j + (size_t)i * lda];
}

template <typename T>
__global__ void mark_kernel(FactorWork<T> w, int *phi) {
    if (ldcg(w.status) != 0) return;
    const int M = min(ldcg(&w.st->n_moved), w.maxmoved);
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        int j = w.moved[m];
        phi[w.lpos[j]] = j;
        w.tmpP[m] = w.perm[j];
    }
}

// Work items of the gather and scatter: for every moved index m whose new position is in the
// trailing block, segments of SEG entries of its trailing line (its L row is permuted at the end).
constexpr int SEG = 1024, IC_THREADS = 256;   // entries per work item, threads of the gather/scatter

__device__ __forceinline__ bool moved_item(long long item, int M, int nt, int *m, int *seg) {
    if (item >= (long long)M * nt) return false;
    *m = (int)(item / nt);
    *seg = (int)(item % nt);
    return true;
}

template <typename T>
__global__ void gather_kernel(FactorWork<T> w, const int *phi) {
    pdl_wait();
    pdl_release();
    if (ldcg(w.status) != 0) return;
    const int M = min(ldcg(&w.st->n_moved), w.maxmoved);
    const int n = w.n, lda = w.lda, kend = w.st->kend;
    const int nt = (n - kend + SEG - 1) / SEG;
    const T *__restrict__ A = w.A;
    int m, seg;
    for (long long item = blockIdx.x; moved_item(item, M, nt, &m, &seg); item += gridDim.x) {
        const int j = w.moved[m], p = w.lpos[j];
        if (p >= kend) {
            // SEG / IC_THREADS entries per thread: their marks, then their entries of A, then the
            // stores (the loads of a thread in flight together)
            T *ta = w.tmpA + (size_t)m * n;
            const int hi = min(n, kend + (seg + 1) * SEG);
            const int q0 = kend + seg * SEG + threadIdx.x;
            int srcq[SEG / IC_THREADS];
            T v[SEG / IC_THREADS];
#pragma unroll
            for (int u = 0; u < SEG / IC_THREADS; ++u) {
                const int q = q0 + u * IC_THREADS;
                srcq[u] = q < hi ? phi[q] : -1;
            }
#pragma unroll
            for (int u = 0; u < SEG / IC_THREADS; ++u) {
                const int q = q0 + u * IC_THREADS;
                if (q < hi) v[u] = a_sym_ld(A, lda, j, srcq[u] >= 0 ? srcq[u] : q);
            }
#pragma unroll
            for (int u = 0; u < SEG / IC_THREADS; ++u) {
                const int q = q0 + u * IC_THREADS;
                if (q < hi) ta[q] = v[u];
            }
        }
    }
}

template <typename T>
__global__ void scatter_kernel(FactorWork<T> w) {
    pdl_wait();
    pdl_release();
    if (ldcg(w.status) != 0) return;
    const int M = min(ldcg(&w.st->n_moved), w.maxmoved);
    const int n = w.n, lda = w.lda, kend = w.st->kend;
    const int nt = (n - kend + SEG - 1) / SEG;
    T *__restrict__ A = w.A;
    int m, seg;
    for (long long item = blockIdx.x; moved_item(item, M, nt, &m, &seg); item += gridDim.x) {
        const int p = w.lpos[w.moved[m]];
        if (p >= kend) {
            const T *ta = w.tmpA + (size_t)m * n;
            const int hi = min(n, kend + (seg + 1) * SEG);
            const int q0 = kend + seg * SEG + threadIdx.x;
            T v[SEG / IC_THREADS];
#pragma unroll
            for (int u = 0; u < SEG / IC_THREADS; ++u) {
                const int q = q0 + u * IC_THREADS;
                if (q < hi) v[u] = ta[q];
            }
#pragma unroll
            for (int u = 0; u < SEG / IC_THREADS; ++u) {
                const int q = q0 + u * IC_THREADS;
                if (q < hi) {
                    if (p >= q) A[(size_t)p + (size_t)q * lda] = v[u];
                    else A[(size_t)q + (size_t)p * lda] = v[u];
                }
            }
        }
    }
}

// Panel multipliers (already in position order, column-major) into A(:, k0:kend); clears the
// position marks.  Work items (column t, chunk x of PS_ROWS rows) over a fixed grid: the panel's
// position is known only on the device, and a grid sized for the whole matrix would launch
// thousands of empty blocks for the late panels.
constexpr int PS_THREADS = 256, PS_ROWS = 4 * PS_THREADS;
template <typename T>
__global__ void __launch_bounds__(PS_THREADS) panel_store_kernel(FactorWork<T> w, int *phi) {
    pdl_wait();
    pdl_release();
    if (ldcg(w.status) != 0) return;
    const int n = w.n, lda = w.lda, k0 = w.st->k0, kend = w.st->kend;
    const int width = kend - k0;
    T *__restrict__ A = w.A;
    // item (t, x): column k0 + t, rows k0 + t + 1 + [x, x + 1) * PS_ROWS
    const int chunks = (n - k0 + PS_ROWS - 1) / PS_ROWS;
    const long long items = width > 0 ? (long long)width * chunks : 0;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int t = (int)(it / chunks), x = (int)(it - (long long)t * chunks);
        const int p0 = k0 + t + 1 + x * PS_ROWS;
        if (p0 >= n) continue;
        const T *__restrict__ src = w.Lc + (size_t)t * n;
        T *__restrict__ dst = A + (size_t)(k0 + t) * lda;
        T v[PS_ROWS / PS_THREADS];
#pragma unroll
        for (int u = 0; u < PS_ROWS / PS_THREADS; ++u) {
            const int p = p0 + u * PS_THREADS + threadIdx.x;
            v[u] = p < n ? src[p] : T(0);
        }
#pragma unroll
        for (int u = 0; u < PS_ROWS / PS_THREADS; ++u) {
            const int p = p0 + u * PS_THREADS + threadIdx.x;
            if (p < n) dst[p] = v[u];
        }
    }
    if (blockIdx.x == 0) {
        const int M = min(w.st->n_moved, w.maxmoved);
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const int j = w.moved[m];
            phi[w.lpos[j]] = -1;
            w.perm[w.lpos[j]] = w.tmpP[m];
        }
    }
}

// ------------------------------------------------------------------------------------------
// Trailing update: A(p, q) -= sum_t W(p, t) L(q, t), kend <= q <= p < n, over the lower
// triangle in TM x TM tiles (persistent loop over the tiles); W rows come from Wbuf
// (column-major, ld n), L21 from the panel columns A(:, k0:kend) just stored.
// ------------------------------------------------------------------------------------------
template <typename T, int TM, int TK, int RM>
__global__ void __launch_bounds__((TM / RM) * (TM / RM))
trailing_simt_kernel(FactorWork<T> w) {
    constexpr int TPR = TM / RM;               // threads along a tile edge
    constexpr int NT = TPR * TPR;
    __shared__ T Wsm[TK][TM];
    __shared__ T Lsm[TK][TM];
    if (ldcg(w.status) != 0) return;
    const int n = w.n, lda = w.lda, k0 = w.st->k0, kend = w.st->kend;
    const int K = kend - k0, N = n - kend;
    if (K <= 0 || N <= 0) return;
    const int nt = (N + TM - 1) / TM;
    const long long total = (long long)nt * (nt + 1) / 2;
    const int tr = threadIdx.x % TPR, tc = threadIdx.x / TPR;
    T *__restrict__ A = w.A;
    const T *__restrict__ W = w.Wbuf;
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int I = (int)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
        while ((long long)I * (I + 1) / 2 > tile) --I;
        while ((long long)(I + 1) * (I + 2) / 2 <= tile) ++I;
        const int J = (int)(tile - (long long)I * (I + 1) / 2);
        const int p0 = kend + I * TM, q0 = kend + J * TM;
        T acc[RM][RM];
#pragma unroll
        for (int a = 0; a < RM; ++a)
#pragma unroll
            for (int b = 0; b < RM; ++b) acc[a][b] = T(0);
        for (int t0 = 0; t0 < K; t0 += TK) {
            for (int e = threadIdx.x; e < TK * TM; e += NT) {
                int r = e % TM, tt = e / TM;
                int p = p0 + r, q = q0 + r, t = t0 + tt;
                bool okt = t < K;
                Wsm[tt][r] = (okt && p < n) ? W[(size_t)p + (size_t)t * n] : T(0);
                Lsm[tt][r] = (okt && q < n) ? A[(size_t)q + (size_t)(k0 + t) * lda] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int tt = 0; tt < TK; ++tt) {
                T a[RM], b[RM];
#pragma unroll
                for (int x = 0; x < RM; ++x) a[x] = Wsm[tt][tr + TPR * x];
#pragma unroll
                for (int x = 0; x < RM; ++x) b[x] = Lsm[tt][tc + TPR * x];
#pragma unroll
                for (int x = 0; x < RM; ++x)
#pragma unroll
                    for (int y = 0; y < RM; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int y = 0; y < RM; ++y) {
            const int q = q0 + tc + TPR * y;
#pragma unroll
            for (int x = 0; x < RM; ++x) {
                const int p = p0 + tr + TPR * x;
                if (p < n && q < n && p >= q) {
                    T *c = A + (size_t)p + (size_t)q * lda;
                    *c = *c - acc[x][y];
                }
            }
        }
    }
}

// marked: the panel kernel already wrote the position marks and saved permutation entries of
// its moved indices (the block QRCP's moved list needs mark_kernel)
template <typename T>
cudaError_t launch_interchange(const FactorWork<T> &w, cudaStream_t s, bool marked) {
    int *phi = w.moved + w.n;   // second half of the moved buffer holds the position marks
    if (!marked) {
        mark_kernel<T><<<1, 256, 0, s>>>(w, phi);
        count_launches(1);
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g = 4 * sms;
    cudaError_t e = launch_pdl(gather_kernel<T>, dim3(g), dim3(IC_THREADS), 0, s, w, (const int *)phi);
    if (e != cudaSuccess) return e;
    count_launches(1);
    e = launch_pdl(scatter_kernel<T>, dim3(g), dim3(IC_THREADS), 0, s, w);
    if (e != cudaSuccess) return e;
    count_launches(1);
    e = launch_pdl(panel_store_kernel<T>, dim3(4 * sms), dim3(PS_THREADS), 0, s, w, phi);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
static int trailing_grid(const void *fn, int threads) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0);
    return sms * (per > 0 ? per : 1);
}

template <>
cudaError_t launch_trailing<double>(const FactorWork<double> &w, int kmin, int mode, cudaStream_t s) {
    (void)mode;
    constexpr int TM = 64, TK = 16, RM = 4;
    static int grid = 0;
    if (!grid) grid = trailing_grid<double>((const void *)trailing_simt_kernel<double, TM, TK, RM>, 256);
    long long nt = (w.n - kmin + TM - 1) / TM;
    long long total = nt * (nt + 1) / 2;
    int g = (int)(total < grid ? (total > 0 ? total : 1) : grid);
    trailing_simt_kernel<double, TM, TK, RM><<<g, (TM / RM) * (TM / RM), 0, s>>>(w);
    count_launches(1);
    return cudaGetLastError();
}

template <>
cudaError_t launch_trailing<float>(const FactorWork<float> &w, int kmin, int mode, cudaStream_t s) {
    if ((mode == 3 || mode == 4) && w.tcops) return launch_trailing_tc(w, w.tcops, kmin, mode == 4, s);   // RCP_TF32X3, RCP_F16X3
    constexpr int TM = 128, TK = 16, RM = 8;
    static int grid = 0;
    if (!grid) grid = trailing_grid<float>((const void *)trailing_simt_kernel<float, TM, TK, RM>, 256);
    long long nt = (w.n - kmin + TM - 1) / TM;
    long long total = nt * (nt + 1) / 2;
    int g = (int)(total < grid ? (total > 0 ? total : 1) : grid);
    trailing_simt_kernel<float, TM, TK, RM><<<g, (TM / RM) * (TM / RM), 0, s>>>(w);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Start and end of a factorization.
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void factor_init_kernel(FactorWork<T> w) {
    const int n = w.n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        FactorState *st = w.st;
        st->next = 0; st->k0 = 0; st->kend = 0; st->info = 0; st->n2x2 = 0; st->n_moved = 0;
        st->beta2 = 0.0; st->min_ratio = 1.0;
        st->maxD_bits = 0ull; st->maxL_bits = 0ull; st->maxA_bits = 0ull;
        st->guard_req = 0; st->guard_k = n; st->nresk = 0; st->rank = n;
    }
    for (int i = tid; i < n; i += gridDim.x * blockDim.x) {
        w.perm[i] = i;
        w.moved[n + i] = -1;       // position marks
        w.Dd[i] = 0.0;
        w.Ds[i] = 0.0;
    }
}

// max |A_ij| over the lower triangle, in the matrix's own type (the maximum of FP32 magnitudes is
// exact in FP32; converting every entry to FP64 would run the pass on the slow FP64 pipe), four
// loads of a thread in flight together
template <typename T>
__global__ void maxabs_lower_kernel(FactorWork<T> w) {
    const int n = w.n, lda = w.lda;
    T m = T(0);
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const T *col = w.A + (size_t)j * lda;
        for (int i0 = j + threadIdx.x; i0 < n; i0 += 4 * blockDim.x) {
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * blockDim.x;
                v[u] = i < n ? col[i] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) m = fmax(m, fabs(v[u]));
        }
    }
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > T(0)) atomic_max_nonneg(&w.st->maxA_bits, (double)m);
}

template <typename T>
__global__ void factor_finish_kernel(FactorWork<T> w) {
    const int n = w.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w.A[(size_t)i + (size_t)i * w.lda] = (T)w.Dd[i];
}

template <typename T>
__global__ void guard_zero_kernel(int n, int k, T *A, int lda, double *Dd, double *Ds) {
    for (int j = k + blockIdx.x; j < n; j += gridDim.x) {
        for (int i = j + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i + (size_t)j * lda] = T(0);
        if (threadIdx.x == 0) {
            Dd[j] = 0.0;
            Ds[j] = 0.0;
        }
    }
}

// perm and the panel bounds after panel blk (after its interchange kernels)
template <typename T>
__global__ void panel_record_kernel(FactorWork<T> w, int blk) {
    pdl_wait();
    pdl_release();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w.pbounds[2 * blk] = w.st->k0;
        w.pbounds[2 * blk + 1] = w.st->kend;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x)
        w.psnap[(size_t)blk * w.n + i] = w.perm[i];
}

template <typename T>
__global__ void perm_inverse_kernel(FactorWork<T> w, int npanels) {
    const long long total = (long long)npanels * w.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int J = (int)(e / w.n), p = (int)(e % w.n);
        const int v = w.psnap[e];
        if ((unsigned)v < (unsigned)w.n) w.pinv[(size_t)J * w.n + v] = p;
    }
}

// Column c of panel J = [k0, kend): the row at final position q >= kend is the row that sat at
// position pinv_J[perm[q]] when panel J ended.  One CTA per column at a time; the column is
// staged in this CTA's slice of the scratch (global, n entries) and gathered back.
template <typename T>
__global__ void lrows_permute_kernel(FactorWork<T> w, int npanels) {
    if (ldcg(w.status) != 0) return;
    const int n = w.n, lda = w.lda;
    T *scr = w.tmpA + (size_t)blockIdx.x * n;
    int J = 0;
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        while (J < npanels && w.pbounds[2 * J + 1] <= c) ++J;
        if (J >= npanels) break;
        const int k0 = w.pbounds[2 * J], kend = w.pbounds[2 * J + 1];
        if (c < k0 || kend >= n) continue;
        const int *inv = w.pinv + (size_t)J * n;
        for (int q = kend + threadIdx.x; q < n; q += blockDim.x) scr[q] = w.A[(size_t)q + (size_t)c * lda];
        __syncthreads();
        for (int q = kend + threadIdx.x; q < n; q += blockDim.x) {
            int src = inv[w.perm[q]];
            if (src < kend || src >= n) src = q;   // cannot happen for a valid record
            w.A[(size_t)q + (size_t)c * lda] = scr[src];
        }
        __syncthreads();
    }
}

// The same permutation with the row map of a panel built once per work unit: a unit is (panel J,
// LP_COLS of its columns); the map q -> pinv_J[perm[q]] of the rows kend..n-1 and one column
// segment at a time sit in shared memory (dynamic: (n - kend) ints + (n - kend) values), so the
// column is read and written in coalesced runs.
constexpr int LP_COLS = 16, LP_THREADS = 512, LP_DEPTH = 16;

template <typename T>
__global__ void __launch_bounds__(LP_THREADS) lrows_permute_smem_kernel(FactorWork<T> w, int npanels) {
    extern __shared__ __align__(16) unsigned char lp_smem[];
    if (ldcg(w.status) != 0) return;
    const int n = w.n, lda = w.lda;
    int nunits = 0;
    for (int J = 0; J < npanels; ++J) nunits += (w.pbounds[2 * J + 1] - w.pbounds[2 * J] + LP_COLS - 1) / LP_COLS;
    int J = 0, ubase = 0;   // units of panels before J
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        int k0 = w.pbounds[2 * J], kend = w.pbounds[2 * J + 1];
        while (u >= ubase + (kend - k0 + LP_COLS - 1) / LP_COLS) {
            ubase += (kend - k0 + LP_COLS - 1) / LP_COLS;
            ++J;
            k0 = w.pbounds[2 * J];
            kend = w.pbounds[2 * J + 1];
        }
        const int m = n - kend;
        if (m <= 0) continue;
        int *map = reinterpret_cast<int *>(lp_smem);
        T *seg = reinterpret_cast<T *>(lp_smem + (((size_t)m * sizeof(int) + 15) & ~(size_t)15));
        const int *inv = w.pinv + (size_t)J * n;
        __syncthreads();   // the previous unit's reads of map and seg are done
        for (int q = threadIdx.x; q < m; q += LP_THREADS) {
            int src = inv[w.perm[kend + q]];
            if (src < kend || src >= n) src = kend + q;   // cannot happen for a valid record
            map[q] = src - kend;
        }
        const int c_lo = k0 + (u - ubase) * LP_COLS, c_hi = min(kend, c_lo + LP_COLS);
        for (int c = c_lo; c < c_hi; ++c) {
            T *col = w.A + (size_t)kend + (size_t)c * lda;
            // LP_DEPTH loads of a thread in flight together before their shared-memory stores
            for (int q0 = threadIdx.x; q0 < m; q0 += LP_THREADS * LP_DEPTH) {
                T v[LP_DEPTH];
#pragma unroll
                for (int u = 0; u < LP_DEPTH; ++u) {
                    const int q = q0 + u * LP_THREADS;
                    v[u] = q < m ? col[q] : T(0);
                }
#pragma unroll
                for (int u = 0; u < LP_DEPTH; ++u) {
                    const int q = q0 + u * LP_THREADS;
                    if (q < m) seg[q] = v[u];
                }
            }
            __syncthreads();
            for (int q = threadIdx.x; q < m; q += LP_THREADS) col[q] = seg[map[q]];
            __syncthreads();
        }
    }
}

template <typename T>
cudaError_t launch_panel_record(const FactorWork<T> &w, int blk, cudaStream_t s) {
    int blocks = (w.n + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    cudaError_t e = launch_pdl(panel_record_kernel<T>, dim3(blocks), dim3(256), 0, s, w, blk);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lrows_permute(const FactorWork<T> &w, int npanels, cudaStream_t s) {
    if (w.n == 0 || npanels <= 0) return cudaSuccess;
    perm_inverse_kernel<T><<<1024, 256, 0, s>>>(w, npanels);
    count_launches(1);
    // rows after the first panel: at most n - 1; map and one column segment in shared memory
    const size_t smem = (((size_t)w.n * sizeof(int) + 15) & ~(size_t)15) + (size_t)w.n * sizeof(T);
    static size_t optin = 0;
    static bool attr[2] = {false, false};
    if (!optin) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        optin = (size_t)v;
    }
    const int ti = sizeof(T) == sizeof(float) ? 0 : 1;
    if (smem <= optin) {
        if (!attr[ti]) {
            // once per type, to the largest size any later call may need
            cudaError_t e = cudaFuncSetAttribute(lrows_permute_smem_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)optin);
            if (e != cudaSuccess) return e;
            attr[ti] = true;
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        lrows_permute_smem_kernel<T><<<sms, LP_THREADS, smem, s>>>(w, npanels);
    } else {
        // grid-stride over columns in increasing order, so each CTA's panel index only advances;
        // the scratch holds maxmoved slices of n entries
        int grid = w.n < w.maxmoved ? w.n : w.maxmoved;
        lrows_permute_kernel<T><<<grid, 256, 0, s>>>(w, npanels);
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_factor_init(const FactorWork<T> &w, cudaStream_t s) {
    int blocks = (w.n + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    factor_init_kernel<T><<<blocks, 256, 0, s>>>(w);
    count_launches(1);
    maxabs_lower_kernel<T><<<w.n < 1024 ? (w.n > 0 ? w.n : 1) : 1024, 256, 0, s>>>(w);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_factor_finish(const FactorWork<T> &w, cudaStream_t s) {
    int blocks = (w.n + 255) / 256;
    if (blocks < 1) blocks = 1;
    factor_finish_kernel<T><<<blocks, 256, 0, s>>>(w);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_guard_zero(int n, int k, T *A, int lda, double *Dd, double *Ds, cudaStream_t s) {
    if (k >= n) return cudaSuccess;
    const int grid = n - k < 1024 ? n - k : 1024;
    guard_zero_kernel<T><<<grid, 256, 0, s>>>(n, k, A, lda, Dd, Ds);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_guard_zero<double>(int, int, double *, int, double *, double *, cudaStream_t);
template cudaError_t launch_guard_zero<float>(int, int, float *, int, double *, double *, cudaStream_t);
template cudaError_t launch_interchange<double>(const FactorWork<double> &, cudaStream_t, bool);
template cudaError_t launch_interchange<float>(const FactorWork<float> &, cudaStream_t, bool);
template cudaError_t launch_panel_record<double>(const FactorWork<double> &, int, cudaStream_t);
template cudaError_t launch_panel_record<float>(const FactorWork<float> &, int, cudaStream_t);
template cudaError_t launch_lrows_permute<double>(const FactorWork<double> &, int, cudaStream_t);
template cudaError_t launch_lrows_permute<float>(const FactorWork<float> &, int, cudaStream_t);
template cudaError_t launch_factor_init<double>(const FactorWork<double> &, cudaStream_t);
template cudaError_t launch_factor_init<float>(const FactorWork<float> &, cudaStream_t);
template cudaError_t launch_factor_finish<double>(const FactorWork<double> &, cudaStream_t);
template cudaError_t launch_factor_finish<float>(const FactorWork<float> &, cudaStream_t);

}  // namespace rcpk
