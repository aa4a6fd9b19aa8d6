// solve.cu -- the solution phase (x = Pi L^{-T} D^+ L^{-1} Pi^T b, the operation-count
// table's "solution phase"; D^+ the pseudo-inverse of D: a zero 1x1 block contributes 0), and
// the FP64 pieces of iterative refinement: the residual r = b - A x with the lower-stored
// original A, ||A||_inf, and the normwise backward error ||r||_inf / (||A||_inf ||x||_inf) of
// the experiments section.  Also one triangle of the solve on its own and ||L||_1, for the
// stability diagnostics (||L||_1, an estimate of ||L^{-1}||_1).
//
// Triangular solves: one persistent launch per triangle.  Row blocks of SV_NB rows are
// handed out in dependency order through an atomic ticket; a block waits (bounded) on the
// "done" flags of the blocks it depends on, subtracts their contributions tile by tile,
// solves its diagonal block one warp per right-hand side, and publishes its flag.
#include <type_traits>

#include "kernels.h"

namespace rcpk {

constexpr int SV_NB = 64, SV_THREADS = 256, SV_RC = 8;

template <typename T>
__device__ __forceinline__ bool wait_flag(const int *flag, int epoch, int *status) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_s32(flag) != epoch) {
            unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_s32(flag) != epoch) {
                if ((++spins & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
                    ok = 0;
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Blocks finish in dependency order (block J is done only after every block it depends on), so
// once the flag of block J is set, warp 0 reads the next 32 flags in one round and returns the
// last block of the finished run: J + m, m = number of consecutive set flags after J, stepping by
// `dir` (+1 forward, -1 backward) and not past `last`.  -1 on a timeout.
__device__ __forceinline__ int wait_run(const int *flags, int J, int last, int dir, int epoch, int *status) {
    __shared__ int s_known;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int ok = 1;
        if (lane == 0 && ld_acquire_s32(flags + J) != epoch) {
            unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_s32(flags + J) != epoch) {
                if ((++spins & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
                    ok = 0;
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        const int j = J + dir * (lane + 1);
        const bool in = dir > 0 ? j <= last : j >= last;
        const bool set = ok && in && ld_acquire_s32(flags + j) == epoch;
        const unsigned bal = __ballot_sync(0xffffffffu, set);
        const int m = bal == 0xffffffffu ? 32 : __ffs(~bal) - 1;
        if (lane == 0) s_known = ok ? J + dir * m : -1;
    }
    __syncthreads();
    return s_known;
}

// acc[r][c] -= sum_jj M(r, jj) y[jj][c] with M given by (Ms, transposed?) in shared memory.
template <typename T, bool TRANS>
__device__ __forceinline__ void block_gemv_sub(T (*acc)[SV_RC], const T (*Ms)[SV_NB + 1], const T (*ys)[SV_RC],
                                               int nr, int nj, int rc) {
    const int pairs = SV_NB * rc;
    const int g = pairs <= 64 ? 4 : (pairs <= 128 ? 2 : 1);
    if (g == 1) {
        for (int e = threadIdx.x; e < pairs; e += SV_THREADS) {
            int r = e % SV_NB, c = e / SV_NB;
            if (r >= nr) continue;
            T s = T(0);
            for (int jj = 0; jj < nj; ++jj) s += (TRANS ? Ms[jj][r] : Ms[r][jj]) * ys[jj][c];
            acc[r][c] -= s;
        }
    } else {
        // split the inner dimension over g threads of the same warp, then reduce
        const int e = threadIdx.x / g, sl = threadIdx.x % g;
        const int r = e % SV_NB, c = e / SV_NB;
        T s = T(0);
        if (r < nr)
            for (int jj = sl; jj < nj; jj += g) s += (TRANS ? Ms[jj][r] : Ms[r][jj]) * ys[jj][c];
        for (int off = g / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (sl == 0 && r < nr) acc[r][c] -= s;
    }
}

// Inverses of the unit lower triangular diagonal blocks L(I, I) (SV_NB x SV_NB, column-major
// at Linv + I * SV_NB * SV_NB; the last block is padded with the identity).  One CTA per block,
// one thread per column: x = L_II^{-1} e_c by forward substitution.
//
// With Mneg / Nneg (the FP32 solves), also the couplings to the neighbouring blocks, negated:
// Mneg_I = -L_II^{-1} L_{I,I-1} (I >= 1) and Nneg_I = -L_{I+1,I} L_II^{-1} (I < nb-1), both
// column-major SV_NB x SV_NB, so that a block's last dependency costs one product:
// y_I = u_I + Mneg_I y_{I-1}, v_I = u_I + Nneg_I^T v_{I+1}.
template <typename T>
__global__ void __launch_bounds__(SV_NB)
inv_diag_kernel(int n, const T *__restrict__ L, int lda, T *Linv, int *status, const int *skip, T *Mneg = nullptr,
                T *Nneg = nullptr) {
    __shared__ T Ls[SV_NB][SV_NB + 1];
    __shared__ T Xs[SV_NB][SV_NB + 1];
    if (skip && ldcg(skip)) return;
    if (ldcg(status) != 0) return;
    const int I = blockIdx.x, r0 = I * SV_NB, nr = min(SV_NB, n - r0);
    const int c = threadIdx.x;
    for (int r = 0; r < SV_NB; ++r)
        Ls[r][c] = (r < nr && c < nr && r > c) ? L[(size_t)(r0 + r) + (size_t)(r0 + c) * lda] : T(0);
    __syncthreads();
    for (int r = 0; r < SV_NB; ++r) Xs[r][c] = r == c ? T(1) : T(0);
    for (int r = c + 1; r < SV_NB; ++r) {
        T s = T(0);
        for (int k = c; k < r; ++k) s = fma(Ls[r][k], Xs[k][c], s);
        Xs[r][c] = -s;
    }
    __syncthreads();
    T *out = Linv + (size_t)I * SV_NB * SV_NB;
    for (int r = 0; r < SV_NB; ++r) out[(size_t)r + (size_t)c * SV_NB] = Xs[r][c];
    const int nb = (n + SV_NB - 1) / SV_NB;
    if (Mneg && I > 0) {
        __syncthreads();   // Ls is read by every column's substitution above
        for (int r = 0; r < SV_NB; ++r)
            Ls[r][c] = r < nr ? L[(size_t)(r0 + r) + (size_t)(r0 - SV_NB + c) * lda] : T(0);   // L_{I,I-1}
        __syncthreads();
        T *m = Mneg + (size_t)I * SV_NB * SV_NB;
        for (int r = 0; r < SV_NB; ++r) {
            T sum = T(0);
            for (int k = 0; k < SV_NB; ++k) sum = fma(Xs[r][k], Ls[k][c], sum);
            m[(size_t)r + (size_t)c * SV_NB] = -sum;
        }
    }
    if (Nneg && I + 1 < nb) {
        const int nr2 = min(SV_NB, n - r0 - SV_NB);
        __syncthreads();
        for (int r = 0; r < SV_NB; ++r)
            Ls[r][c] = (r < nr2 && c < nr) ? L[(size_t)(r0 + SV_NB + r) + (size_t)(r0 + c) * lda] : T(0);   // L_{I+1,I}
        __syncthreads();
        T *m = Nneg + (size_t)I * SV_NB * SV_NB;
        for (int jj = 0; jj < SV_NB; ++jj) {
            T sum = T(0);
            for (int k = 0; k < SV_NB; ++k) sum = fma(Ls[jj][k], Xs[k][c], sum);
            m[(size_t)jj + (size_t)c * SV_NB] = -sum;
        }
    }
}

// A SV_NB x SV_NB tile of L, column-major with leading dimension lda, staged through registers:
// every thread holds TILE_PER_THREAD entries (issued as independent loads).
constexpr int TILE_PER_THREAD = SV_NB * SV_NB / SV_THREADS;

template <typename T>
__device__ __forceinline__ void tile_load(T (&reg)[TILE_PER_THREAD], const T *__restrict__ L, int lda, int r0, int c0,
                                          int nr, int nc) {
#pragma unroll
    for (int u = 0; u < TILE_PER_THREAD; ++u) {
        const int e = threadIdx.x + u * SV_THREADS;
        const int r = e % SV_NB, cc = e / SV_NB;
        reg[u] = (r < nr && cc < nc) ? L[(size_t)(r0 + r) + (size_t)(c0 + cc) * lda] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void tile_store(const T (&reg)[TILE_PER_THREAD], T (*Ms)[SV_NB + 1]) {
#pragma unroll
    for (int u = 0; u < TILE_PER_THREAD; ++u) {
        const int e = threadIdx.x + u * SV_THREADS;
        Ms[e % SV_NB][e / SV_NB] = reg[u];
    }
}

// y of one finished block (SV_NB x SV_RC, rows past nj and columns past rc zero) through
// registers, so that it can be loaded a tile ahead.
constexpr int YS_PER_THREAD = SV_NB * SV_RC / SV_THREADS;

template <typename T>
__device__ __forceinline__ void ys_load(T (&reg)[YS_PER_THREAD], const T *Y, int n, int j0, int nj, int c0, int rc) {
#pragma unroll
    for (int u = 0; u < YS_PER_THREAD; ++u) {
        const int e = threadIdx.x + u * SV_THREADS;
        const int jj = e % SV_NB, c = e / SV_NB;
        reg[u] = (jj < nj && c < rc) ? ldcg(Y + (size_t)(j0 + jj) + (size_t)(c0 + c) * n) : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void ys_store(const T (&reg)[YS_PER_THREAD], T (*ys)[SV_RC]) {
#pragma unroll
    for (int u = 0; u < YS_PER_THREAD; ++u) {
        const int e = threadIdx.x + u * SV_THREADS;
        ys[e % SV_NB][e / SV_NB] = reg[u];
    }
}

// Forward: L y = Pi^T x (L unit lower).  Y (work, type T, n x nrhs, ld n) receives y.  The next
// tile of L is loaded into registers before the flag of the block it multiplies is awaited, and
// the diagonal block is applied through its precomputed inverse (a GEMV, not a sequential sweep).
template <typename T>
__global__ void __launch_bounds__(SV_THREADS)
fwd_kernel(int n, int nrhs, const T *__restrict__ L, int lda, const T *__restrict__ Linv,
           const int *__restrict__ perm, const double *__restrict__ X, int ldx, T *Y, int *flags, int epoch,
           int *ticket, int *status, const int *skip) {
    __shared__ T Ms[SV_NB][SV_NB + 1];
    __shared__ T acc[SV_NB][SV_RC];
    __shared__ T ys[SV_NB][SV_RC];
    __shared__ int s_I;
    if (skip && ldcg(skip)) return;
    if (ldcg(status) != 0) return;
    const int nb = (n + SV_NB - 1) / SV_NB;
    for (;;) {
        if (threadIdx.x == 0) s_I = atomicAdd(ticket, 1);
        __syncthreads();
        const int I = s_I;
        __syncthreads();
        if (I >= nb) return;
        const int r0 = I * SV_NB, nr = min(SV_NB, n - r0);
        for (int c0 = 0; c0 < nrhs; c0 += SV_RC) {
            const int rc = min(SV_RC, nrhs - c0);
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                acc[r][c] = (r < nr && c < rc) ? (T)X[(size_t)perm[r0 + r] + (size_t)(c0 + c) * ldx] : T(0);
            }
            // the inverse of the diagonal block, needed last, is loaded first
            T lreg[TILE_PER_THREAD];
            tile_load(lreg, Linv + (size_t)I * SV_NB * SV_NB, SV_NB, 0, 0, SV_NB, SV_NB);
            T cur[TILE_PER_THREAD], nxt[TILE_PER_THREAD];
            T ysr[YS_PER_THREAD];   // y of the next finished block, prefetched
            bool have = false;
            int known = -1;         // every block <= known is finished
            if (I > 0) tile_load(cur, L, lda, r0, 0, nr, SV_NB);
            for (int J = 0; J < I; ++J) {
                if (J + 1 < I) tile_load(nxt, L, lda, r0, (J + 1) * SV_NB, nr, SV_NB);
                tile_store(cur, Ms);
                if (J > known) {
                    known = wait_run(flags, J, I - 1, 1, epoch, status);
                    if (known < 0) return;
                }
                if (!have) ys_load<T>(ysr, Y, n, J * SV_NB, SV_NB, c0, rc);
                ys_store<T>(ysr, ys);
                have = J + 1 < I && J + 1 <= known;
                if (have) ys_load<T>(ysr, Y, n, (J + 1) * SV_NB, SV_NB, c0, rc);
                __syncthreads();
                block_gemv_sub<T, false>(acc, Ms, ys, nr, SV_NB, rc);
                __syncthreads();
#pragma unroll
                for (int u = 0; u < TILE_PER_THREAD; ++u) cur[u] = nxt[u];
            }
            // y_I = L_II^{-1} acc
            tile_store(lreg, Ms);
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                ys[r][c] = acc[r][c];
                acc[r][c] = T(0);
            }
            __syncthreads();
            block_gemv_sub<T, false>(acc, Ms, ys, nr, nr, rc);   // acc = -Linv * y
            __syncthreads();
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                if (r < nr && c < rc) stcg(Y + (size_t)(r0 + r) + (size_t)(c0 + c) * n, -acc[r][c]);
            }
            __syncthreads();
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release_s32(flags + I, epoch);
    }
}

// Block-diagonal solve D w = y in place (FP64 arithmetic for the 2x2 blocks).
template <typename T>
__global__ void dsolve_kernel(int n, int nrhs, const double *__restrict__ Dd, const double *__restrict__ Ds,
                              T *Y, int *status, const int *skip) {
    if (skip && ldcg(skip)) return;
    if (ldcg(status) != 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i > 0 && Ds[i - 1] != 0.0) continue;       // second row of a 2x2 block
        if (i + 1 < n && Ds[i] != 0.0) {
            const double b = Ds[i], a = Dd[i] / b, c = Dd[i + 1] / b, den = a * c - 1.0;
            for (int k = 0; k < nrhs; ++k) {
                T *y = Y + (size_t)k * n;
                double y1 = (double)y[i] / b, y2 = (double)y[i + 1] / b;
                y[i] = (T)((c * y1 - y2) / den);
                y[i + 1] = (T)((a * y2 - y1) / den);
            }
        } else {
            // a zero 1x1 block (exact singularity, or the Schur complement where the safeguard
            // stopped) contributes 0: the pseudo-inverse of D, i.e. the basic solution
            const double dv = Dd[i];
            for (int k = 0; k < nrhs; ++k)
                Y[(size_t)i + (size_t)k * n] = (T)(dv != 0.0 ? (double)Y[(size_t)i + (size_t)k * n] / dv : 0.0);
        }
    }
}

// Backward: L^T v = w, then X(perm[i], :) = v(i, :).  Blocks are taken last to first; the
// diagonal block goes through the transpose of its precomputed inverse.
template <typename T>
__global__ void __launch_bounds__(SV_THREADS)
bwd_kernel(int n, int nrhs, const T *__restrict__ L, int lda, const T *__restrict__ Linv,
           const int *__restrict__ perm, double *X, int ldx, T *Y, int *flags, int epoch, int *ticket, int *status,
           const int *skip) {
    __shared__ T Ms[SV_NB][SV_NB + 1];
    __shared__ T acc[SV_NB][SV_RC];
    __shared__ T ys[SV_NB][SV_RC];
    __shared__ int s_I;
    if (skip && ldcg(skip)) return;
    if (ldcg(status) != 0) return;
    const int nb = (n + SV_NB - 1) / SV_NB;
    for (;;) {
        if (threadIdx.x == 0) s_I = atomicAdd(ticket, 1);
        __syncthreads();
        const int It = s_I;
        __syncthreads();
        if (It >= nb) return;
        const int I = nb - 1 - It;
        const int r0 = I * SV_NB, nr = min(SV_NB, n - r0);
        for (int c0 = 0; c0 < nrhs; c0 += SV_RC) {
            const int rc = min(SV_RC, nrhs - c0);
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                acc[r][c] = (r < nr && c < rc) ? ldcg(Y + (size_t)(r0 + r) + (size_t)(c0 + c) * n) : T(0);
            }
            // tiles L(J, I) for J = nb-1 down to I+1, Ms[jj][r] = L(j0 + jj, r0 + r)
            T lreg[TILE_PER_THREAD];
            tile_load(lreg, Linv + (size_t)I * SV_NB * SV_NB, SV_NB, 0, 0, SV_NB, SV_NB);
            T cur[TILE_PER_THREAD], nxt[TILE_PER_THREAD];
            T ysr[YS_PER_THREAD];
            bool have = false;
            int known = nb;         // every block >= known is finished
            if (I + 1 < nb) tile_load(cur, L, lda, (nb - 1) * SV_NB, r0, min(SV_NB, n - (nb - 1) * SV_NB), nr);
            for (int J = nb - 1; J > I; --J) {
                if (J - 1 > I) tile_load(nxt, L, lda, (J - 1) * SV_NB, r0, min(SV_NB, n - (J - 1) * SV_NB), nr);
                tile_store(cur, Ms);
                if (J < known) {
                    known = wait_run(flags, J, I + 1, -1, epoch, status);
                    if (known < 0) return;
                }
                const int j0 = J * SV_NB, nj = min(SV_NB, n - j0);
                if (!have) ys_load<T>(ysr, Y, n, j0, nj, c0, rc);
                ys_store<T>(ysr, ys);
                have = J - 1 > I && J - 1 >= known;
                if (have) ys_load<T>(ysr, Y, n, (J - 1) * SV_NB, min(SV_NB, n - (J - 1) * SV_NB), c0, rc);
                __syncthreads();
                block_gemv_sub<T, true>(acc, Ms, ys, nr, nj, rc);
                __syncthreads();
#pragma unroll
                for (int u = 0; u < TILE_PER_THREAD; ++u) cur[u] = nxt[u];
            }
            // v_I = (L_II^{-1})^T acc: Ms[jj][r] = Linv(jj, r) used transposed
            tile_store(lreg, Ms);
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                ys[r][c] = acc[r][c];
                acc[r][c] = T(0);
            }
            __syncthreads();
            block_gemv_sub<T, true>(acc, Ms, ys, nr, nr, rc);   // acc = -Linv^T * w
            __syncthreads();
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                if (r < nr && c < rc) {
                    const T v = -acc[r][c];
                    stcg(Y + (size_t)(r0 + r) + (size_t)(c0 + c) * n, v);
                    X[(size_t)perm[r0 + r] + (size_t)(c0 + c) * ldx] = (double)v;
                }
            }
            __syncthreads();
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release_s32(flags + I, epoch);
    }
}

// ------------------------------------------------------------------------------------------
// FP32 triangular solves with self-validating results.  Every entry of a finished block is
// published as one 64-bit word (epoch << 32 | float bits) with a single relaxed store, and a
// reader polls the words it needs until their epoch is the current one: the poll returns the
// data itself, so a block's result reaches the blocks below it in one L2 round trip, without a
// separate flag, fence or second load.  The words of the next finished block are requested a
// tile ahead; a block re-polls only the words that were not yet current.  Epochs start at 1 and
// the buffers are zeroed when allocated, so a word never matches before it is written.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void st_word(unsigned long long *p, float v, int epoch) {
    const unsigned long long w = ((unsigned long long)(unsigned)epoch << 32) | __float_as_uint(v);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long *p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

// request the words of rows j0 .. j0+nj-1 (columns c0 .. c0+rc-1); entries outside are 0 and
// marked current
__device__ __forceinline__ void words_issue(unsigned long long (&w)[YS_PER_THREAD], const unsigned long long *Yp, int n,
                                            int j0, int nj, int c0, int rc, int epoch) {
#pragma unroll
    for (int u = 0; u < YS_PER_THREAD; ++u) {
        const int e = threadIdx.x + u * SV_THREADS;
        const int jj = e % SV_NB, c = e / SV_NB;
        w[u] = (jj < nj && c < rc) ? ld_word(Yp + (size_t)(j0 + jj) + (size_t)(c0 + c) * n)
                                   : (unsigned long long)(unsigned)epoch << 32;
    }
}

// wait until every requested word is current (bounded), then stage the values; false to every
// thread of the CTA when any thread's wait ran out
__device__ __forceinline__ bool words_stage(unsigned long long (&w)[YS_PER_THREAD], const unsigned long long *Yp, int n,
                                            int j0, int c0, int epoch, float (*ys)[SV_RC], int *status) {
    int ok = 1;
#pragma unroll
    for (int u = 0; u < YS_PER_THREAD; ++u) {
        if ((int)(w[u] >> 32) != epoch) {
            const int e = threadIdx.x + u * SV_THREADS;
            const unsigned long long *p = Yp + (size_t)(j0 + e % SV_NB) + (size_t)(c0 + e / SV_NB) * n;
            const unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while ((int)((w[u] = ld_word(p)) >> 32) != epoch) {
                if ((++spins & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
                    ok = 0;
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
            }
        }
        const int e = threadIdx.x + u * SV_THREADS;
        ys[e % SV_NB][e / SV_NB] = __uint_as_float((unsigned)w[u]);
    }
    return __syncthreads_and(ok) != 0;
}

// Forward: L y = Pi^T x, y published as words in Yp (n x nrhs, ld n).  Every finished block but
// the last enters through its tile of L; then u = L_II^{-1} acc, and the last block through
// y_I = u + Mneg_I y_{I-1} (its words were requested a tile ahead).
__global__ void __launch_bounds__(SV_THREADS)
fwd_words_kernel(int n, int nrhs, const float *__restrict__ L, int lda, const float *__restrict__ Linv,
                 const float *__restrict__ Mneg, const int *__restrict__ perm, const double *__restrict__ X, int ldx,
                 unsigned long long *Yp, int epoch, int *ticket, int *status, const int *skip) {
    __shared__ float Ms[SV_NB][SV_NB + 1];
    __shared__ float acc[SV_NB][SV_RC];
    __shared__ float ys[SV_NB][SV_RC];
    __shared__ int s_I;
    if (skip && ldcg(skip)) return;
    if (ldcg(status) != 0) return;
    const int nb = (n + SV_NB - 1) / SV_NB;
    for (;;) {
        if (threadIdx.x == 0) s_I = atomicAdd(ticket, 1);
        __syncthreads();
        const int I = s_I;
        __syncthreads();
        if (I >= nb) return;
        const int r0 = I * SV_NB, nr = min(SV_NB, n - r0);
        for (int c0 = 0; c0 < nrhs; c0 += SV_RC) {
            const int rc = min(SV_RC, nrhs - c0);
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                acc[r][c] = (r < nr && c < rc) ? (float)X[(size_t)perm[r0 + r] + (size_t)(c0 + c) * ldx] : 0.f;
            }
            float lreg[TILE_PER_THREAD], mreg[TILE_PER_THREAD];
            tile_load(lreg, Linv + (size_t)I * SV_NB * SV_NB, SV_NB, 0, 0, SV_NB, SV_NB);
            if (I > 0) tile_load(mreg, Mneg + (size_t)I * SV_NB * SV_NB, SV_NB, 0, 0, SV_NB, SV_NB);
            float cur[TILE_PER_THREAD], nxt[TILE_PER_THREAD];
            unsigned long long wr[YS_PER_THREAD];
            if (I > 0) {
                if (I >= 2) tile_load(cur, L, lda, r0, 0, nr, SV_NB);
                words_issue(wr, Yp, n, 0, SV_NB, c0, rc, epoch);
            }
            for (int J = 0; J + 1 < I; ++J) {
                if (J + 2 < I) tile_load(nxt, L, lda, r0, (J + 1) * SV_NB, nr, SV_NB);
                tile_store(cur, Ms);
                if (!words_stage(wr, Yp, n, J * SV_NB, c0, epoch, ys, status)) return;
                words_issue(wr, Yp, n, (J + 1) * SV_NB, SV_NB, c0, rc, epoch);
                block_gemv_sub<float, false>(acc, Ms, ys, nr, SV_NB, rc);
                __syncthreads();
#pragma unroll
                for (int u = 0; u < TILE_PER_THREAD; ++u) cur[u] = nxt[u];
            }
            // u = L_II^{-1} acc, before the last finished block is awaited
            tile_store(lreg, Ms);
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                ys[r][c] = acc[r][c];
                acc[r][c] = 0.f;
            }
            __syncthreads();
            block_gemv_sub<float, false>(acc, Ms, ys, nr, nr, rc);   // acc = -u
            __syncthreads();
            if (I > 0) {
                tile_store(mreg, Ms);
                if (!words_stage(wr, Yp, n, (I - 1) * SV_NB, c0, epoch, ys, status)) return;
                block_gemv_sub<float, false>(acc, Ms, ys, nr, SV_NB, rc);   // acc = -u - Mneg y_{I-1} = -y_I
                __syncthreads();
            }
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                if (r < nr && c < rc) st_word(Yp + (size_t)(r0 + r) + (size_t)(c0 + c) * n, -acc[r][c], epoch);
            }
            __syncthreads();
        }
    }
}

// Block-diagonal solve D w = y (FP64 arithmetic for the 2x2 blocks), from the words of the
// forward solve into the plain array W.
__global__ void dsolve_words_kernel(int n, int nrhs, const double *__restrict__ Dd, const double *__restrict__ Ds,
                                    const unsigned long long *__restrict__ Yp, float *W, int *status, const int *skip) {
    if (skip && ldcg(skip)) return;
    if (ldcg(status) != 0) return;
    auto yv = [&](int i, int k) { return (double)__uint_as_float((unsigned)ldcg(Yp + (size_t)i + (size_t)k * n)); };
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i > 0 && Ds[i - 1] != 0.0) continue;       // second row of a 2x2 block
        if (i + 1 < n && Ds[i] != 0.0) {
            const double b = Ds[i], a = Dd[i] / b, c = Dd[i + 1] / b, den = a * c - 1.0;
            for (int k = 0; k < nrhs; ++k) {
                const double y1 = yv(i, k) / b, y2 = yv(i + 1, k) / b;
                W[(size_t)i + (size_t)k * n] = (float)((c * y1 - y2) / den);
                W[(size_t)i + 1 + (size_t)k * n] = (float)((a * y2 - y1) / den);
            }
        } else {
            const double dv = Dd[i];   // zero 1x1 block: pseudo-inverse 0
            for (int k = 0; k < nrhs; ++k) W[(size_t)i + (size_t)k * n] = (float)(dv != 0.0 ? yv(i, k) / dv : 0.0);
        }
    }
}

// Backward: L^T v = w (w from W), v published as words in Vp, X(perm[i], :) = v(i, :).  Every
// finished block but the last (I + 1) enters through its tile of L; then u = L_II^{-T} acc, and
// v_I = u + Nneg_I^T v_{I+1}.
__global__ void __launch_bounds__(SV_THREADS)
bwd_words_kernel(int n, int nrhs, const float *__restrict__ L, int lda, const float *__restrict__ Linv,
                 const float *__restrict__ Nneg, const int *__restrict__ perm, double *X, int ldx,
                 const float *__restrict__ W, unsigned long long *Vp, int epoch, int *ticket, int *status,
                 const int *skip) {
    __shared__ float Ms[SV_NB][SV_NB + 1];
    __shared__ float acc[SV_NB][SV_RC];
    __shared__ float ys[SV_NB][SV_RC];
    __shared__ int s_I;
    if (skip && ldcg(skip)) return;
    if (ldcg(status) != 0) return;
    const int nb = (n + SV_NB - 1) / SV_NB;
    for (;;) {
        if (threadIdx.x == 0) s_I = atomicAdd(ticket, 1);
        __syncthreads();
        const int It = s_I;
        __syncthreads();
        if (It >= nb) return;
        const int I = nb - 1 - It;
        const int r0 = I * SV_NB, nr = min(SV_NB, n - r0);
        for (int c0 = 0; c0 < nrhs; c0 += SV_RC) {
            const int rc = min(SV_RC, nrhs - c0);
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                acc[r][c] = (r < nr && c < rc) ? W[(size_t)(r0 + r) + (size_t)(c0 + c) * n] : 0.f;
            }
            // tiles L(J, I) for J = nb-1 down to I+2, Ms[jj][r] = L(j0 + jj, r0 + r)
            float lreg[TILE_PER_THREAD], nreg[TILE_PER_THREAD];
            tile_load(lreg, Linv + (size_t)I * SV_NB * SV_NB, SV_NB, 0, 0, SV_NB, SV_NB);
            if (I + 1 < nb) tile_load(nreg, Nneg + (size_t)I * SV_NB * SV_NB, SV_NB, 0, 0, SV_NB, SV_NB);
            float cur[TILE_PER_THREAD], nxt[TILE_PER_THREAD];
            unsigned long long wr[YS_PER_THREAD];
            if (I + 1 < nb) {
                const int jl = (nb - 1) * SV_NB;
                if (I + 2 < nb) tile_load(cur, L, lda, jl, r0, min(SV_NB, n - jl), nr);
                words_issue(wr, Vp, n, jl, min(SV_NB, n - jl), c0, rc, epoch);
            }
            for (int J = nb - 1; J > I + 1; --J) {
                if (J - 1 > I + 1) tile_load(nxt, L, lda, (J - 1) * SV_NB, r0, min(SV_NB, n - (J - 1) * SV_NB), nr);
                tile_store(cur, Ms);
                const int j0 = J * SV_NB, nj = min(SV_NB, n - j0);
                if (!words_stage(wr, Vp, n, j0, c0, epoch, ys, status)) return;
                words_issue(wr, Vp, n, (J - 1) * SV_NB, min(SV_NB, n - (J - 1) * SV_NB), c0, rc, epoch);
                block_gemv_sub<float, true>(acc, Ms, ys, nr, nj, rc);
                __syncthreads();
#pragma unroll
                for (int u = 0; u < TILE_PER_THREAD; ++u) cur[u] = nxt[u];
            }
            // u = L_II^{-T} acc, before the last finished block is awaited
            tile_store(lreg, Ms);
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                ys[r][c] = acc[r][c];
                acc[r][c] = 0.f;
            }
            __syncthreads();
            block_gemv_sub<float, true>(acc, Ms, ys, nr, nr, rc);   // acc = -u
            __syncthreads();
            if (I + 1 < nb) {
                tile_store(nreg, Ms);
                const int j0 = (I + 1) * SV_NB, nj = min(SV_NB, n - j0);
                if (!words_stage(wr, Vp, n, j0, c0, epoch, ys, status)) return;
                block_gemv_sub<float, true>(acc, Ms, ys, nr, nj, rc);   // acc = -u - Nneg^T v_{I+1} = -v_I
                __syncthreads();
            }
            for (int e = threadIdx.x; e < SV_NB * SV_RC; e += SV_THREADS) {
                int r = e % SV_NB, c = e / SV_NB;
                if (r < nr && c < rc) {
                    const float v = -acc[r][c];
                    st_word(Vp + (size_t)(r0 + r) + (size_t)(c0 + c) * n, v, epoch);
                    X[(size_t)perm[r0 + r] + (size_t)(c0 + c) * ldx] = (double)v;
                }
            }
            __syncthreads();
        }
    }
}

// Work layout (solve_work_bytes).  FP64: T Y[n * nrhs] (rounded up to 256 bytes), then
// T Linv[nb * NB * NB]; flags: int[2 * nb] (forward, backward), then the two tickets.  FP32:
// u64 Yp[n * nrhs], u64 Vp[n * nrhs], float W[n * nrhs] (rounded up to 256 bytes), then
// float Linv[nb * NB * NB]; of the flags only the two tickets are used.  The caller zeroes the
// work area when it is allocated.
// Epoch of a solve launch: the flags and published words of the work area carry it, so every
// launcher that uses the area takes it from this one counter (a reused value would make stale
// entries look current).
static int next_solve_epoch() {
    static int epoch = 0;
    epoch = epoch % 1000000000 + 1;
    return epoch;
}

template <typename T>
static size_t solve_vec_bytes(int n, int nrhs) {
    const size_t v = ((size_t)n * nrhs * sizeof(T) + 255) / 256 * 256;
    return std::is_same<T, float>::value ? 2 * (size_t)n * nrhs * sizeof(unsigned long long) + v : v;
}

template <typename T>
size_t solve_work_bytes(int n, int nrhs) {
    const size_t nb = ((size_t)n + SV_NB - 1) / SV_NB;
    // the inverted diagonal blocks; FP32 also the negated couplings Mneg, Nneg
    const size_t mats = std::is_same<T, float>::value ? 3 : 1;
    return solve_vec_bytes<T>(n, nrhs) + mats * nb * SV_NB * SV_NB * sizeof(T);
}

template <typename T>
cudaError_t launch_solve(int n, int nrhs, const T *L, int lda, const double *Dd, const double *Ds,
                         const int *perm, double *X, int ldx, T *work, int *flags, int *status,
                         const int *skip, cudaStream_t s, bool reuse_inv) {
    if (n == 0 || nrhs == 0) return cudaSuccess;
    const int epoch = next_solve_epoch();
    const int nb = (n + SV_NB - 1) / SV_NB;
    int *tickets = flags + 2 * nb;
    T *Linv = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(work) + solve_vec_bytes<T>(n, nrhs));
    cudaError_t e = cudaMemsetAsync(tickets, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nb < sms ? nb : sms;
    if constexpr (std::is_same<T, float>::value) {
        float *Mneg = Linv + (size_t)nb * SV_NB * SV_NB, *Nneg = Mneg + (size_t)nb * SV_NB * SV_NB;
        if (!reuse_inv) {
            inv_diag_kernel<T><<<nb, SV_NB, 0, s>>>(n, L, lda, Linv, status, skip, Mneg, Nneg);
            count_launches(1);
        }
        unsigned long long *Yp = reinterpret_cast<unsigned long long *>(work);
        unsigned long long *Vp = Yp + (size_t)n * nrhs;
        float *W = reinterpret_cast<float *>(Vp + (size_t)n * nrhs);
        fwd_words_kernel<<<grid, SV_THREADS, 0, s>>>(n, nrhs, L, lda, Linv, Mneg, perm, X, ldx, Yp, epoch, tickets,
                                                     status, skip);
        count_launches(1);
        dsolve_words_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, nrhs, Dd, Ds, Yp, W, status, skip);
        count_launches(1);
        bwd_words_kernel<<<grid, SV_THREADS, 0, s>>>(n, nrhs, L, lda, Linv, Nneg, perm, X, ldx, W, Vp, epoch,
                                                     tickets + 1, status, skip);
        count_launches(1);
    } else {
        if (!reuse_inv) {
            inv_diag_kernel<T><<<nb, SV_NB, 0, s>>>(n, L, lda, Linv, status, skip);
            count_launches(1);
        }
        T *Y = work;
        fwd_kernel<T><<<grid, SV_THREADS, 0, s>>>(n, nrhs, L, lda, Linv, perm, X, ldx, Y, flags, epoch, tickets, status,
                                                  skip);
        count_launches(1);
        dsolve_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(n, nrhs, Dd, Ds, Y, status, skip);
        count_launches(1);
        bwd_kernel<T><<<grid, SV_THREADS, 0, s>>>(n, nrhs, L, lda, Linv, perm, X, ldx, Y, flags + nb, epoch,
                                                  tickets + 1, status, skip);
        count_launches(1);
    }
    return cudaGetLastError();
}

// ---- one triangle of the solve on its own (1-norm estimate of L^{-1}) ----
__global__ void words_to_double_kernel(int n, const unsigned long long *Yp, double *x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = (double)__uint_as_float((unsigned)ldcg(Yp + i));
}

__global__ void double_to_float_kernel(int n, const double *x, float *w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w[i] = (float)x[i];
}

__global__ void iota_kernel(int n, int *p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

cudaError_t launch_iota(int n, int *p, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    iota_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(n, p);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tri_solve(int n, const T *L, int lda, const int *iperm, double *x, T *work, int *flags,
                             int *status, int mode, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int epoch = next_solve_epoch();
    const int nb = (n + SV_NB - 1) / SV_NB;
    int *tickets = flags + 2 * nb;
    T *Linv = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(work) + solve_vec_bytes<T>(n, 1));
    cudaError_t e = cudaMemsetAsync(tickets, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nb < sms ? nb : sms, vgrid = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    if constexpr (std::is_same<T, float>::value) {
        float *Mneg = Linv + (size_t)nb * SV_NB * SV_NB, *Nneg = Mneg + (size_t)nb * SV_NB * SV_NB;
        inv_diag_kernel<T><<<nb, SV_NB, 0, s>>>(n, L, lda, Linv, status, nullptr, Mneg, Nneg);
        unsigned long long *Yp = reinterpret_cast<unsigned long long *>(work);
        unsigned long long *Vp = Yp + (size_t)n;
        float *W = reinterpret_cast<float *>(Vp + (size_t)n);
        if (mode == 0) {
            fwd_words_kernel<<<grid, SV_THREADS, 0, s>>>(n, 1, L, lda, Linv, Mneg, iperm, x, n, Yp, epoch, tickets,
                                                         status, nullptr);
            words_to_double_kernel<<<vgrid, 256, 0, s>>>(n, Yp, x);
        } else {
            double_to_float_kernel<<<vgrid, 256, 0, s>>>(n, x, W);
            bwd_words_kernel<<<grid, SV_THREADS, 0, s>>>(n, 1, L, lda, Linv, Nneg, iperm, x, n, W, Vp, epoch,
                                                         tickets + 1, status, nullptr);
        }
        count_launches(3);
    } else {
        inv_diag_kernel<T><<<nb, SV_NB, 0, s>>>(n, L, lda, Linv, status, nullptr);
        T *Y = work;
        if (mode == 0) {
            fwd_kernel<T><<<grid, SV_THREADS, 0, s>>>(n, 1, L, lda, Linv, iperm, x, n, Y, flags, epoch, tickets, status,
                                                      nullptr);
            e = cudaMemcpyAsync(x, Y, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
        } else {
            e = cudaMemcpyAsync(Y, x, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
            bwd_kernel<T><<<grid, SV_THREADS, 0, s>>>(n, 1, L, lda, Linv, iperm, x, n, Y, flags + nb, epoch,
                                                      tickets + 1, status, nullptr);
        }
        count_launches(2);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// ||L||_1 of the unit lower L: max over columns of 1 + sum_{i > j} |L(i, j)|
template <typename T>
__global__ void __launch_bounds__(256) l_norm1_kernel(int n, const T *__restrict__ L, int lda, unsigned long long *out) {
    __shared__ double red[8];
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        double s = 0.0;
        for (int i = j + 1 + (int)threadIdx.x; i < n; i += 256) s += fabs((double)L[(size_t)i + (size_t)j * lda]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 1.0;
            for (int q = 0; q < 8; ++q) t += red[q];
            atomic_max_nonneg(out, t);
        }
        __syncthreads();
    }
}

template <typename T>
cudaError_t launch_l_norm1(int n, const T *L, int lda, unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n <= 0) return e;
    l_norm1_kernel<T><<<n < 1216 ? n : 1216, 256, 0, s>>>(n, L, lda, out);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_tri_solve<double>(int, const double *, int, const int *, double *, double *, int *, int *,
                                              int, cudaStream_t);
template cudaError_t launch_tri_solve<float>(int, const float *, int, const int *, double *, float *, int *, int *,
                                             int, cudaStream_t);
template cudaError_t launch_l_norm1<double>(int, const double *, int, unsigned long long *, cudaStream_t);
template cudaError_t launch_l_norm1<float>(int, const float *, int, unsigned long long *, cudaStream_t);
template size_t solve_work_bytes<double>(int, int);
template size_t solve_work_bytes<float>(int, int);
template cudaError_t launch_solve<double>(int, int, const double *, int, const double *, const double *, const int *,
                                          double *, int, double *, int *, int *, const int *, cudaStream_t, bool);
template cudaError_t launch_solve<float>(int, int, const float *, int, const double *, const double *, const int *,
                                         double *, int, float *, int *, int *, const int *, cudaStream_t, bool);

// ------------------------------------------------------------------------------------------
// Refinement pieces (FP64).
// ------------------------------------------------------------------------------------------
constexpr int RV_ROWS = 64, RV_CW = 1024;   // row block and column chunk of the row pass

// Row pass: part[ch][c][i] = sum_{j in chunk ch, j <= i} A(i, j) x_j   (ABS: |A(i, j)|, x = 1)
template <bool ABS>
__global__ void __launch_bounds__(256)
symv_rows_kernel(int n, int nrhs, const double *__restrict__ A, int lda, const double *__restrict__ X, int ldx,
                 double *part, const int *skip) {
    if (skip && ldcg(skip)) return;
    const int r0 = blockIdx.x * RV_ROWS, ch = blockIdx.y;
    const int jlo = ch * RV_CW;
    const int r = threadIdx.x % RV_ROWS, sl = threadIdx.x / RV_ROWS;   // 4 column slices
    const int i = r0 + r;
    const int jhi = min(min(n, jlo + RV_CW), r0 + RV_ROWS);
    __shared__ double red[4][RV_ROWS];
    for (int c = 0; c < (ABS ? 1 : nrhs); ++c) {
        double s = 0.0;
        if (i < n) {
            const double *xc = X ? X + (size_t)c * ldx : nullptr;
            for (int j = jlo + sl; j < jhi; j += 4) {
                if (j > i) break;
                double a = A[(size_t)i + (size_t)j * lda];
                s += ABS ? fabs(a) : a * xc[j];
            }
        }
        red[sl][r] = s;
        __syncthreads();
        if (sl == 0 && i < n)
            part[((size_t)ch * (ABS ? 1 : nrhs) + c) * n + i] = red[0][r] + red[1][r] + red[2][r] + red[3][r];
        __syncthreads();
    }
}

// Column pass: y2[c][j] = sum_{i > j} A(i, j) x_i  (one warp per column)
template <bool ABS>
__global__ void symv_cols_kernel(int n, int nrhs, const double *__restrict__ A, int lda,
                                 const double *__restrict__ X, int ldx, double *y2, const int *skip) {
    if (skip && ldcg(skip)) return;
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= n) return;
    const double *col = A + (size_t)j * lda;
    for (int c = 0; c < (ABS ? 1 : nrhs); ++c) {
        const double *xc = X ? X + (size_t)c * ldx : nullptr;
        double s = 0.0;
        for (int i = j + 1 + lane; i < n; i += 32) s += ABS ? fabs(col[i]) : col[i] * xc[i];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) y2[(size_t)c * n + j] = s;
    }
}

// R = B - (sum_ch part + y2); per-column max |r| and max |x| into mx[2*c], mx[2*c+1] (bits).
__global__ void residual_combine_kernel(int n, int nrhs, int nch, const double *part, const double *y2,
                                        const double *__restrict__ Bv, int ldb, const double *__restrict__ X,
                                        int ldx, double *R, int ldr, unsigned long long *mx, const int *skip) {
    if (skip && ldcg(skip)) return;
    for (int c = 0; c < nrhs; ++c) {
        double rm = 0.0, xm = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            double y = y2[(size_t)c * n + i];
            for (int ch = 0; ch < nch; ++ch) y += part[((size_t)ch * nrhs + c) * n + i];
            double r = Bv[(size_t)i + (size_t)c * ldb] - y;
            R[(size_t)i + (size_t)c * ldr] = r;
            rm = fmax(rm, fabs(r));
            xm = fmax(xm, fabs(X[(size_t)i + (size_t)c * ldx]));
        }
        for (int off = 16; off > 0; off >>= 1) {
            rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, off));
            xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, off));
        }
        if ((threadIdx.x & 31) == 0) {
            if (rm > 0.0 || isnan(rm)) atomicMax(mx + 2 * c, (unsigned long long)__double_as_longlong(isnan(rm) ? INFINITY : rm));
            if (xm > 0.0) atomicMax(mx + 2 * c + 1, (unsigned long long)__double_as_longlong(xm));
        }
    }
}

__global__ void anorm_finish_kernel(int n, int nch, const double *part, const double *y2, double *anorm) {
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double y = y2[i];
        for (int ch = 0; ch < nch; ++ch) y += part[(size_t)ch * n + i];
        m = fmax(m, y);
    }
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) v = fmax(v, red[w]);
        *anorm = v;
    }
}

// berr = max_c ||r_c||_inf / (||A||_inf ||x_c||_inf); sets conv when berr <= tol.
__global__ void refine_check_kernel(int nrhs, const unsigned long long *mx, const double *anorm, double tol,
                                    int *conv, double *berr, double *prev, int *iters, int count_iter) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (*conv) return;
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        double rm = __longlong_as_double((long long)mx[2 * c]), xm = __longlong_as_double((long long)mx[2 * c + 1]);
        double e = (*anorm > 0.0 && xm > 0.0) ? rm / (*anorm * xm) : (rm > 0.0 ? INFINITY : 0.0);
        if (!(e <= worst)) worst = e;
    }
    *berr = worst;
    if (worst <= tol) *conv = 1;
    else if (*prev > 0.0 && !(worst <= 0.5 * *prev)) *conv = 2;   // the last correction did not halve berr
    else if (count_iter) *iters += 1;
    *prev = worst;
}

__global__ void axpy_kernel(int n, int nrhs, double *X, int ldx, const double *D, int ldd, const int *skip) {
    if (skip && ldcg(skip)) return;
    long long total = (long long)n * nrhs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % n), c = (int)(e / n);
        X[(size_t)i + (size_t)c * ldx] += D[(size_t)i + (size_t)c * ldd];
    }
}

static int nchunks(int n) { return (n + RV_CW - 1) / RV_CW; }

// part: >= symv_part_doubles(n, nrhs) doubles; mx: 2*nrhs u64 maxima
size_t symv_part_doubles(int n, int nrhs) { return ((size_t)nchunks(n) + 1) * (size_t)nrhs * (size_t)n + 64; }

cudaError_t launch_symv_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                                 const double *Bv, int ldb, double *R, int ldr, double *part,
                                 unsigned long long *mx, const int *skip, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int nch = nchunks(n);
    double *y2 = part + (size_t)nch * nrhs * n;
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * 2 * nrhs, s);
    if (e != cudaSuccess) return e;
    dim3 g((n + RV_ROWS - 1) / RV_ROWS, nch);
    symv_rows_kernel<false><<<g, 256, 0, s>>>(n, nrhs, A, lda, X, ldx, part, skip);
    count_launches(1);
    symv_cols_kernel<false><<<(n + 7) / 8, 256, 0, s>>>(n, nrhs, A, lda, X, ldx, y2, skip);
    count_launches(1);
    int blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    residual_combine_kernel<<<blocks, 256, 0, s>>>(n, nrhs, nch, part, y2, Bv, ldb, X, ldx, R, ldr, mx, skip);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_anorm(int n, const double *A, int lda, double *part, double *anorm, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(anorm, 0, sizeof(double), s);
    const int nch = nchunks(n);
    double *y2 = part + (size_t)nch * n;
    dim3 g((n + RV_ROWS - 1) / RV_ROWS, nch);
    symv_rows_kernel<true><<<g, 256, 0, s>>>(n, 1, A, lda, nullptr, 0, part, nullptr);
    count_launches(1);
    symv_cols_kernel<true><<<(n + 7) / 8, 256, 0, s>>>(n, 1, A, lda, nullptr, 0, y2, nullptr);
    count_launches(1);
    anorm_finish_kernel<<<1, 1024, 0, s>>>(n, nch, part, y2, anorm);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_refine_check(int nrhs, const unsigned long long *mx, const double *anorm, double tol, int *conv,
                                double *berr, double *prev, int *iters, int count_iter, cudaStream_t s) {
    refine_check_kernel<<<1, 32, 0, s>>>(nrhs, mx, anorm, tol, conv, berr, prev, iters, count_iter);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_axpy_update(int n, int nrhs, double *X, int ldx, const double *D, int ldd, const int *skip,
                               cudaStream_t s) {
    long long total = (long long)n * nrhs;
    if (total == 0) return cudaSuccess;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    axpy_kernel<<<blocks, 256, 0, s>>>(n, nrhs, X, ldx, D, ldd, skip);
    count_launches(1);
    return cudaGetLastError();
}

// Copy of the lower triangle of an FP64 matrix (columns c0 .. c1-1), optionally rounded to FP32.
__global__ void copy_lower_kernel(int n, const double *__restrict__ src, int lds, void *dst, int ldd, int to_f32, int c0,
                                  int c1) {
    // four loads of a thread in flight together before their stores
    for (int j = c0 + blockIdx.x; j < c1; j += gridDim.x) {
        const double *sc = src + (size_t)j * lds;
        for (int i0 = j + threadIdx.x; i0 < n; i0 += 4 * blockDim.x) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * blockDim.x;
                v[u] = i < n ? sc[i] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < n) {
                    if (to_f32) static_cast<float *>(dst)[(size_t)i + (size_t)j * ldd] = (float)v[u];
                    else static_cast<double *>(dst)[(size_t)i + (size_t)j * ldd] = v[u];
                }
            }
        }
    }
}

cudaError_t launch_copy_lower_f64(int n, const double *src, int lds, void *dst, int ldd, int to_f32, cudaStream_t s,
                                  int c0, int c1) {
    if (c1 < 0) c1 = n;
    if (n == 0 || c1 <= c0) return cudaSuccess;
    const int cols = c1 - c0;
    copy_lower_kernel<<<cols < 4096 ? cols : 4096, 256, 0, s>>>(n, src, lds, dst, ldd, to_f32, c0, c1);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rcpk
