// sketch.cu -- the Gaussian sketch of Section 3: Omega (d x n, entries N(0,1)) drawn from
// Philox4x64-10 (Salmon et al., SC'11) through Box-Muller, and the random projection
// B = Omega A of the lower-stored symmetric A.
//
// Omega is drawn once into workspace (d*n values; FP64 transcendental throughput on this
// part is too low to redraw it inside every GEMM tile) and stays L2-resident for the GEMM.
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

// One thread per pair (2t, 2t+1) of column j: counter (j, t, 0, 0), key (seed, 0).
template <typename T>
__global__ void omega_kernel(int d, int n, uint64_t seed, T *__restrict__ om) {
    const int half = (d + 1) / 2;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)half * n) return;
    int j = (int)(idx / half), t = (int)(idx % half);
    uint64_t x[4] = {(uint64_t)j, (uint64_t)t, 0ull, 0ull};
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

template <typename T>
cudaError_t launch_omega(int d, int n, uint64_t seed, T *om, cudaStream_t s) {
    long long total = (long long)((d + 1) / 2) * n;
    if (total == 0) return cudaSuccess;
    int blocks = (int)((total + 255) / 256);
    omega_kernel<T><<<blocks, 256, 0, s>>>(d, n, seed, om);
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
cudaError_t launch_sketch(int n, int d, const TA *A, int lda, const TC *om, TC *B, float *A32,
                          int lda32, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (d < 1 || d > 16 * SK_MAXRPT) return cudaErrorInvalidValue;
    return launch_sketch_rpt<TA, TC>(n, d, A, lda, om, B, A32, lda32, s);
}

template cudaError_t launch_omega<double>(int, int, uint64_t, double *, cudaStream_t);
template cudaError_t launch_omega<float>(int, int, uint64_t, float *, cudaStream_t);
template cudaError_t launch_sketch<double, double>(int, int, const double *, int, const double *, double *,
                                                   float *, int, cudaStream_t);
template cudaError_t launch_sketch<double, float>(int, int, const double *, int, const float *, float *,
                                                  float *, int, cudaStream_t);
template cudaError_t launch_sketch<float, float>(int, int, const float *, int, const float *, float *,
                                                 float *, int, cudaStream_t);

}  // namespace rcpk
