// gmres.cu -- FP64 vector kernels of GMRES-based iterative refinement.
//
// Classic iterative refinement (x += solve(r), with the backward error of the experiments
// section as its stopping test) converges only while the factor's error times the condition
// number stays below one.  For harder systems the
// correction equation A d = r is solved instead by GMRES (Saad and Schultz, 1986) on the
// preconditioned operator M^{-1} A, M = the computed L D L^T (Carson and Higham, 2017/2018:
// "GMRES-based iterative refinement").  Every vector of that iteration is FP64 and
// n-long; the operator applications reuse the FP64 SYMV of the residual and the triangular
// solves.  What remains are the Krylov basis operations below: dot products against the
// basis (deterministic: per-block partial sums, then a fixed-order sum per column), the
// Gram-Schmidt update w -= V h, and scaling.
#include "kernels.h"

namespace rcpk {

constexpr int GM_THREADS = 256;
constexpr int GM_ROWS = 8192;   // rows per block of a dot product

// part[c * nb + blk] = sum over block blk's rows i of V(i, c) w(i), c < ncol
__global__ void __launch_bounds__(GM_THREADS) gm_dots_kernel(int n, const double *__restrict__ V, int ldv,
                                                             const double *__restrict__ w, double *part, int nb) {
    __shared__ double red[GM_THREADS / 32];
    const int c = blockIdx.y, blk = blockIdx.x;
    const int i0 = blk * GM_ROWS, i1 = min(n, i0 + GM_ROWS);
    const double *v = V + (size_t)c * ldv;
    double s = 0.0;
    for (int i = i0 + (int)threadIdx.x; i < i1; i += GM_THREADS) s = fma(v[i], w[i], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < GM_THREADS / 32; ++q) t += red[q];
        part[(size_t)c * nb + blk] = t;
    }
}

// out[c] = sum over blocks of part[c * nb + blk], one warp per column, fixed order
__global__ void gm_dots_finish_kernel(int nb, const double *part, double *out) {
    const int c = blockIdx.x, lane = threadIdx.x;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += part[(size_t)c * nb + b];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[c] = s;
}

// w(i) += sign * sum_{c < ncol} V(i, c) h(c)
__global__ void __launch_bounds__(GM_THREADS) gm_update_kernel(int n, int ncol, const double *__restrict__ V, int ldv,
                                                               const double *__restrict__ h, double sign, double *w) {
    for (int i = blockIdx.x * GM_THREADS + threadIdx.x; i < n; i += gridDim.x * GM_THREADS) {
        double s = 0.0;
        for (int c = 0; c < ncol; ++c) s = fma(V[(size_t)i + (size_t)c * ldv], h[c], s);
        w[i] = fma(sign, s, w[i]);
    }
}

__global__ void __launch_bounds__(GM_THREADS) gm_scale_kernel(int n, double f, double *w) {
    for (int i = blockIdx.x * GM_THREADS + threadIdx.x; i < n; i += gridDim.x * GM_THREADS) w[i] *= f;
}

static int gm_blocks(int n) { return (n + GM_ROWS - 1) / GM_ROWS; }

static int gm_grid(int n) {
    const int b = (n + GM_THREADS - 1) / GM_THREADS;
    return b < 1216 ? (b > 0 ? b : 1) : 1216;   // 8 blocks per SM on 152 SMs
}

size_t gm_part_doubles(int n, int ncol_max) { return (size_t)gm_blocks(n) * (size_t)ncol_max + 8; }

cudaError_t launch_gm_dots(int n, int ncol, const double *V, int ldv, const double *w, double *part, double *out,
                           cudaStream_t s) {
    if (ncol <= 0) return cudaSuccess;
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(double) * ncol, s);
    const int nb = gm_blocks(n);
    gm_dots_kernel<<<dim3(nb, ncol), GM_THREADS, 0, s>>>(n, V, ldv, w, part, nb);
    count_launches(1);
    gm_dots_finish_kernel<<<ncol, 32, 0, s>>>(nb, part, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gm_update(int n, int ncol, const double *V, int ldv, const double *h, double sign, double *w,
                             cudaStream_t s) {
    if (n <= 0 || ncol <= 0) return cudaSuccess;
    gm_update_kernel<<<gm_grid(n), GM_THREADS, 0, s>>>(n, ncol, V, ldv, h, sign, w);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gm_scale(int n, double f, double *w, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    gm_scale_kernel<<<gm_grid(n), GM_THREADS, 0, s>>>(n, f, w);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rcpk
