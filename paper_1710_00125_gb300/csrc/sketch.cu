// sketch.cu -- the Gaussian sketch of Section 3: Omega (d x n, entries N(0,1)) drawn from
// Philox4x64-10 (Salmon et al., SC'11) through Box-Muller, and the random projection
// B = Omega A of the lower-stored symmetric A.
//
// Omega is drawn once into workspace (d*n values; FP64 transcendental throughput on this
// part is too low to redraw it inside every GEMM tile) and stays L2-resident for the GEMM.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace rcpk {

__device__ __forceinline__ void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
        uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
        uint64_t y0 = hi1 ^ x[1] ^ k0;
        uint64_t y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
        k0 += W0; k1 += W1;
    }
}

// One thread per pair (2t, 2t+1) of column j: counter (j, t, stream, 0), key (seed, 0).
template <typename T>
__global__ void omega_kernel(int d, int n, uint64_t seed, uint64_t stream, T *__restrict__ om) {
    const int half = (d + 1) / 2;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)half * n) return;
    int j = (int)(idx / half), t = (int)(idx % half);
    uint64_t x[4] = {(uint64_t)j, (uint64_t)t, stream, 0ull};
    philox4x64_10(x, seed, 0ull);
    double u1 = ((double)(x[0] >> 11) + 1.0) * 0x1.0p-53;
    double u2 = (double)(x[1] >> 11) * 0x1.0p-53;
    double rho = sqrt(-2.0 * log(u1));
    double th = 6.283185307179586476925286766559 * u2;
    double s, c;
    sincos(th, &s, &c);
    om[(size_t)2 * t + (size_t)j * d] = (T)(rho * c);
    if (2 * t + 1 < d) om[(size_t)2 * t + 1 + (size_t)j * d] = (T)(rho * s);
}

// B(:, J) = sum_I Omega(:, I) A(I, J) for a 64-column block J per CTA; A(I, J) comes from
// the stored lower triangle directly (I >= J) or transposed (I < J).  TA is the stored type
// of A, TC the arithmetic type (= type of Omega and B).  When A32 != nullptr the CTA also
// writes the FP32 rounding of the lower tiles it owns (tiles (I, J) with I >= J).
constexpr int SK_BJ = 64, SK_BK = 32, SK_THREADS = 256, SK_MAXRPT = 8;   // d <= 128

template <typename TA, typename TC, int RPT>
__global__ void __launch_bounds__(SK_THREADS)
sketch_kernel(int n, int d, const TA *__restrict__ A, int lda, const TC *__restrict__ om,
              TC *__restrict__ B, float *__restrict__ A32, int lda32) {
    __shared__ TC Os[SK_BK][16 * RPT];
    __shared__ __align__(16) TC As[SK_BK][SK_BJ];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int j0 = blockIdx.x * SK_BJ;
    TC acc[RPT][4];
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[u][c] = TC(0);

    for (int i0 = 0; i0 < n; i0 += SK_BK) {
        // Omega(0:d, i0:i0+BK) -> Os[ii][r]
        for (int e = threadIdx.x; e < SK_BK * 16 * RPT; e += SK_THREADS) {
            int ii = e / (16 * RPT), r = e % (16 * RPT);
            int i = i0 + ii;
            Os[ii][r] = (r < d && i < n) ? om[(size_t)r + (size_t)i * d] : TC(0);
        }
        // A_sym(i0:i0+BK, j0:j0+BJ) -> As[ii][jj]
        const bool below = i0 >= j0 + SK_BJ, above = i0 + SK_BK <= j0;
        if (below) {
            for (int e = threadIdx.x; e < SK_BK * SK_BJ; e += SK_THREADS) {
                int ii = e % SK_BK, jj = e / SK_BK;
                int i = i0 + ii, j = j0 + jj;
                TA v = (i < n && j < n) ? A[(size_t)i + (size_t)j * lda] : TA(0);
                As[ii][jj] = (TC)v;
                if (A32 && i < n && j < n) A32[(size_t)i + (size_t)j * lda32] = (float)v;
            }
        } else if (above) {
            for (int e = threadIdx.x; e < SK_BK * SK_BJ; e += SK_THREADS) {
                int jj = e % SK_BJ, ii = e / SK_BJ;
                int i = i0 + ii, j = j0 + jj;
                As[ii][jj] = (i < n && j < n) ? (TC)A[(size_t)j + (size_t)i * lda] : TC(0);
            }
        } else {
            for (int e = threadIdx.x; e < SK_BK * SK_BJ; e += SK_THREADS) {
                int ii = e % SK_BK, jj = e / SK_BK;
                int i = i0 + ii, j = j0 + jj;
                TC v = TC(0);
                if (i < n && j < n) {
                    if (i >= j) {
                        TA a = A[(size_t)i + (size_t)j * lda];
                        v = (TC)a;
                        if (A32) A32[(size_t)i + (size_t)j * lda32] = (float)a;
                    } else {
                        v = (TC)A[(size_t)j + (size_t)i * lda];
                    }
                }
                As[ii][jj] = v;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int ii = 0; ii < SK_BK; ++ii) {
            TC a[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) a[c] = As[ii][tx * 4 + c];
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                TC o = Os[ii][ty + 16 * u];
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[u][c] = fma(o, a[c], acc[u][c]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        int r = ty + 16 * u;
        if (r >= d) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int j = j0 + tx * 4 + c;
            if (j < n) B[(size_t)r + (size_t)j * d] = acc[u][c];
        }
    }
}

// FP32 sketch, B(:, J) = sum over K slices of Omega(:, I) A(I, J): work units of 128 columns
// x one K slice, spread evenly over a persistent grid; with S > 1 slices each unit writes its
// partial sum to scratch and sketch_reduce_kernel adds the S partials in slice order (the
// result does not depend on the schedule).  Per K step of 32 rows the next tiles are loaded
// into registers while the current ones are used; the A tile sits in shared memory with its
// 16-byte slots XOR-swizzled by row (slot c of row k at c ^ (k & 7)), so that both the
// transposing stores of tiles below the diagonal (8 rows x 4 columns per warp) and the
// straight stores of tiles above it (32 columns of one row) hit 32 distinct banks.  Each
// thread accumulates RPT rows of Omega (ty + 16 u) x 8 consecutive columns (tx * 8 + c).
constexpr int SKF_BJ = 128, SKF_BK = 32, SKF_THREADS = 256;

template <int RPT>
__global__ void __launch_bounds__(SKF_THREADS, RPT <= 5 ? 2 : 1)
sketch_f32_kernel(int n, int d, const float *__restrict__ A, int lda, const float *__restrict__ om,
                  float *__restrict__ out, int S, int Jb, int ksteps, int c0, int c1) {
    constexpr int DP = 16 * RPT;                          // Omega rows, padded
    constexpr int AV = SKF_BK * SKF_BJ / SKF_THREADS;     // A values staged per thread (16)
    constexpr int OV = SKF_BK * DP / SKF_THREADS;         // Omega values staged per thread
    static_assert(AV == 16 && (SKF_BK * DP) % SKF_THREADS == 0, "tile shape");
    __shared__ __align__(16) float As[SKF_BK][SKF_BJ];
    __shared__ float Os[SKF_BK][DP];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, wid = tid >> 5;
    const int units = Jb * S;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int jb = u % Jb, sl = u / Jb;
        const int j0 = c0 + jb * SKF_BJ;   // columns c0 .. c1-1 of B (A is read in columns < c1 only)
        const int kb = (int)((long long)ksteps * sl / S), ke = (int)((long long)ksteps * (sl + 1) / S);
        float acc[RPT][8];
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
        float ra[AV], ro[OV];
        int kind = 0;   // of the staged tile: 0 below the diagonal or mixed, 1 above
        auto fetch = [&](int ks) {
            const int i0 = ks * SKF_BK;
            kind = (i0 + SKF_BK <= j0) ? 1 : 0;
            if (kind == 1) {
                // A(i, j) = A[j + i lda]: 32 consecutive columns of one row per warp
#pragma unroll
                for (int v = 0; v < AV; ++v) {
                    const int j = j0 + lane + 32 * (v & 3), i = i0 + wid + 8 * (v >> 2);
                    ra[v] = (i < n && j < c1) ? A[(size_t)j + (size_t)i * lda] : 0.f;
                }
            } else {
                // 8 consecutive rows x 4 columns per warp (32-byte segments of the stored columns)
                const bool below = i0 >= j0 + SKF_BJ;
#pragma unroll
                for (int v = 0; v < AV; ++v) {
                    const int i = i0 + (lane & 7) + 8 * (v & 3);
                    const int j = j0 + (lane >> 3) + 4 * wid + 32 * (v >> 2);
                    float x = 0.f;
                    if (i < n && j < c1) x = (below || i >= j) ? A[(size_t)i + (size_t)j * lda] : A[(size_t)j + (size_t)i * lda];
                    ra[v] = x;
                }
            }
#pragma unroll
            for (int v = 0; v < OV; ++v) {
                const int e = tid + SKF_THREADS * v, k = e / DP, r = e - k * DP;
                ro[v] = (r < d && i0 + k < n) ? om[(size_t)r + (size_t)(i0 + k) * d] : 0.f;
            }
        };
        auto stage = [&]() {
#pragma unroll
            for (int v = 0; v < AV; ++v) {
                int k, j;
                if (kind == 1) { j = lane + 32 * (v & 3); k = wid + 8 * (v >> 2); }
                else { k = (lane & 7) + 8 * (v & 3); j = (lane >> 3) + 4 * wid + 32 * (v >> 2); }
                As[k][4 * ((j >> 2) ^ (k & 7)) + (j & 3)] = ra[v];
            }
#pragma unroll
            for (int v = 0; v < OV; ++v) {
                const int e = tid + SKF_THREADS * v, k = e / DP, r = e - k * DP;
                Os[k][r] = ro[v];
            }
        };
        if (kb < ke) fetch(kb);
        for (int ks = kb; ks < ke; ++ks) {
            __syncthreads();   // the previous step's reads of As / Os are done
            stage();
            __syncthreads();
            if (ks + 1 < ke) fetch(ks + 1);
#pragma unroll 4
            for (int k = 0; k < SKF_BK; ++k) {
                const float4 *row = reinterpret_cast<const float4 *>(&As[k][0]);
                const float4 a0 = row[(2 * tx) ^ (k & 7)], a1 = row[(2 * tx + 1) ^ (k & 7)];
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const float o = Os[k][ty + 16 * r];
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(o, a[c], acc[r][c]);
                }
            }
        }
        // out holds the columns c0 .. c1-1 (slice sl of S)
        float *dst = out + (size_t)sl * d * (c1 - c0);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int row = ty + 16 * r;
            if (row >= d) continue;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = j0 + tx * 8 + c;
                if (j < c1) dst[(size_t)row + (size_t)(j - c0) * d] = acc[r][c];
            }
        }
    }
}

// B = sum_{s < S} part[s] (slice order), d x n
__global__ void sketch_reduce_kernel(size_t count, int S, const float *__restrict__ part, float *__restrict__ B) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        float v = part[e];
        for (int s = 1; s < S; ++s) v += part[(size_t)s * count + e];
        B[e] = v;
    }
}

cudaError_t launch_sketch_reduce(size_t count, int S, const float *part, float *B, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int blocks = (int)std::min<size_t>((count + 255) / 256, 4096);
    sketch_reduce_kernel<<<blocks, 256, 0, s>>>(count, S, part, B);
    count_launches(1);
    return cudaGetLastError();
}

template <int RPT>
static int sketch_f32_grid() {
    static int g = 0;
    if (g == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sketch_f32_kernel<RPT>, SKF_THREADS, 0);
        g = sms * (per > 0 ? per : 1);
    }
    return g;
}

// K slices of the FP32 sketch: a function of n alone (8 K steps of 32 rows or more per slice, at
// most 64 slices), so that every column is summed in the same slices and order whichever columns
// a launch covers (the whole sketch, or one block of columns as it arrives from the host)
static int sketch_slices(int n) {
    const int ksteps = (n + SKF_BK - 1) / SKF_BK;
    return std::max(1, std::min(64, ksteps / 8));
}

size_t sketch_scratch_floats(int n, int d) {
    const int S = sketch_slices(n);
    return S > 1 ? (size_t)S * d * n : 0;
}

static cudaError_t launch_sketch_f32(int n, int d, const float *A, int lda, const float *om, float *B, float *part,
                                     size_t part_floats, int c0, int c1, cudaStream_t s) {
    const int rpt = (d + 15) / 16;
    int grid = 0;
    switch (rpt) {
#define SKF_G(R) case R: grid = sketch_f32_grid<R>(); break;
        SKF_G(1) SKF_G(2) SKF_G(3) SKF_G(4) SKF_G(5) SKF_G(6) SKF_G(7) SKF_G(8)
#undef SKF_G
        default: return cudaErrorInvalidValue;
    }
    const int nc = c1 - c0;
    const int Jb = (nc + SKF_BJ - 1) / SKF_BJ, ksteps = (n + SKF_BK - 1) / SKF_BK;
    const int S = sketch_slices(n);
    if (S > 1 && (!part || part_floats < (size_t)S * d * nc)) return cudaErrorInvalidValue;   // scratch too small
    float *out = S > 1 ? part : B + (size_t)c0 * d;
    grid = std::min(grid, Jb * S);
    switch (rpt) {
#define SKF_CASE(R) case R: sketch_f32_kernel<R><<<grid, SKF_THREADS, 0, s>>>(n, d, A, lda, om, out, S, Jb, ksteps, c0, c1); break;
        SKF_CASE(1) SKF_CASE(2) SKF_CASE(3) SKF_CASE(4) SKF_CASE(5) SKF_CASE(6) SKF_CASE(7) SKF_CASE(8)
#undef SKF_CASE
    }
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (S > 1) return launch_sketch_reduce((size_t)d * nc, S, part, B + (size_t)c0 * d, s);
    return cudaSuccess;
}

cudaError_t launch_sketch_cols_f32(int n, int d, const float *A, int lda, const float *om, float *B, float *part,
                                   size_t part_floats, int c0, int c1, cudaStream_t s) {
    if (n == 0 || c1 <= c0) return cudaSuccess;
    if (d < 1 || d > 16 * SK_MAXRPT || c0 < 0 || c1 > n) return cudaErrorInvalidValue;
    return launch_sketch_f32(n, d, A, lda, om, B, part, part_floats, c0, c1, s);
}

template <typename T>
cudaError_t launch_omega(int d, int n, uint64_t seed, T *om, cudaStream_t s, uint64_t stream) {
    long long total = (long long)((d + 1) / 2) * n;
    if (total == 0) return cudaSuccess;
    int blocks = (int)((total + 255) / 256);
    omega_kernel<T><<<blocks, 256, 0, s>>>(d, n, seed, stream, om);
    count_launches(1);
    return cudaGetLastError();
}

template <typename TA, typename TC>
static cudaError_t launch_sketch_rpt(int n, int d, const TA *A, int lda, const TC *om, TC *B,
                                     float *A32, int lda32, cudaStream_t s) {
    int grid = (n + SK_BJ - 1) / SK_BJ;
    int rpt = (d + 15) / 16;
    switch (rpt) {
#define SK_CASE(R) case R: sketch_kernel<TA, TC, R><<<grid, SK_THREADS, 0, s>>>(n, d, A, lda, om, B, A32, lda32); break;
        SK_CASE(1) SK_CASE(2) SK_CASE(3) SK_CASE(4) SK_CASE(5) SK_CASE(6) SK_CASE(7) SK_CASE(8)
#undef SK_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename TA, typename TC>
cudaError_t launch_sketch(int n, int d, const TA *A, int lda, const TC *om, TC *B, TC *part, size_t part_elems,
                          cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (d < 1 || d > 16 * SK_MAXRPT) return cudaErrorInvalidValue;
    if constexpr (std::is_same<TA, float>::value && std::is_same<TC, float>::value)
        return launch_sketch_f32(n, d, A, lda, om, B, part, part_elems, 0, n, s);
    return launch_sketch_rpt<TA, TC>(n, d, A, lda, om, B, nullptr, 0, s);
}

template cudaError_t launch_omega<double>(int, int, uint64_t, double *, cudaStream_t, uint64_t);
template cudaError_t launch_omega<float>(int, int, uint64_t, float *, cudaStream_t, uint64_t);
template cudaError_t launch_sketch<double, double>(int, int, const double *, int, const double *, double *,
                                                   double *, size_t, cudaStream_t);
template cudaError_t launch_sketch<float, float>(int, int, const float *, int, const float *, float *, float *,
                                                 size_t, cudaStream_t);

}  // namespace rcpk
