// noalloc.cu -- rcp_solve_noalloc: the solution phase without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a solve: hard real-time
// loops that must never block in the allocator, and programs whose device memory is entirely
// owned by another allocator (a framework's pool, an embedding application with a fixed
// budget).  For them this entry point runs the same forward / block-diagonal / backward kernels
// as rcp_solve, but takes its scratch (the work vector, the row-block flags, the tickets and a
// status word) from one statically sized __device__ array instead of a handle's cudaMalloc'ed
// workspace.
//
// That array lives in every GPU that loads this library until the process exits.  All calls
// share it: two calls whose kernels overlap on the GPU (different streams, or different host
// threads on one stream without ordering) race on it and give wrong results.
#include <algorithm>
#include <mutex>

#include "../../include/rcp.h"
#include "kernels.h"

namespace {

// 16 MiB of scratch: the solve's work area, then 2 * ceil(n / 64) + 2 flag/ticket words and one
// status word.  Work area (nb = ceil(n / 64)): FP64 factors, the work vector (8 n nrhs bytes,
// rounded up to 256) and the inverted 64 x 64 diagonal blocks of L (8 * 4096 nb bytes); FP32
// factors, two arrays of 64-bit (epoch, value) words (16 n nrhs bytes), an FP32 vector (4 n nrhs
// bytes, rounded up to 256) and three 64 x 64 FP32 matrices per row block (12 * 4096 nb bytes).
constexpr size_t kScratchBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_solve_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.  In
// host code the symbol is only a host-side stand-in; its device address must come from the
// runtime with the device current.
void *scratch_address(rcp_status *err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        *err = RCP_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_solve_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            *err = RCP_ECUDA;
            return nullptr;
        }
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

size_t work_bytes(int n, int nrhs, bool f64) {
    const size_t w = f64 ? rcpk::solve_work_bytes<double>(n, nrhs) : rcpk::solve_work_bytes<float>(n, nrhs);
    return (w + 255) / 256 * 256;
}

size_t scratch_needed(int n, int nrhs, bool f64) {
    const size_t nb = ((size_t)n + 63) / 64;
    return work_bytes(n, nrhs, f64) + (2 * nb + 2 + 1) * sizeof(int);
}

// A solve whose device status word is set (a bounded wait that ran out, a non-finite diagonal
// block) has no valid result: its solutions are overwritten with NaN, so that the failure is
// visible in X (this entry point has no handle to report it through).
__global__ void poison_on_status_kernel(int n, int nrhs, double *X, int ldx, const int *status) {
    if (*(volatile const int *)status == 0) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const long long total = (long long)n * nrhs;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        X[(size_t)(e % n) + (size_t)(e / n) * ldx] = nan;
}

}  // namespace

extern "C" rcp_status rcp_solve_noalloc(int n, int nrhs, const void *LA, int lda, const double *Dd,
                                        const double *Ds, const int *perm, rcp_prec prec, double *X,
                                        int ldx, rcp_stream_t stream) {
    if (n < 0 || nrhs < 0 || prec < RCP_FP64 || prec > RCP_F16X3) return RCP_EINVAL;
    if (n == 0 || nrhs == 0) return RCP_OK;
    if (!LA || !Dd || !Ds || !perm || !X || lda < n || ldx < n) return RCP_EINVAL;
    const bool f64 = prec == RCP_FP64;
    if (scratch_needed(n, nrhs, f64) > kScratchBytes) return RCP_EUNSUPPORTED;
    rcp_status err = RCP_OK;
    unsigned char *base = static_cast<unsigned char *>(scratch_address(&err));
    if (!base) return err;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = ((size_t)n + 63) / 64;
    int *flags = reinterpret_cast<int *>(base + work_bytes(n, nrhs, f64));   // 2*nb flags, then 2 tickets
    int *status = flags + 2 * nb + 2;
    // The flags, tickets and status word must start at zero for this call: earlier calls left
    // their epochs and tickets behind.
    if (cudaMemsetAsync(flags, 0, (2 * nb + 3) * sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return RCP_ECUDA;
    }
    // FP32 factors: a reader takes a 64-bit word of the two word arrays as published once its
    // high half equals the call's epoch.  Whatever an earlier call left there (words of another
    // size, doubles of an FP64 solve) could match by chance, so the word arrays start at zero.
    if (!f64 && cudaMemsetAsync(base, 0, 2 * (size_t)n * nrhs * sizeof(unsigned long long), s) != cudaSuccess) {
        cudaGetLastError();
        return RCP_ECUDA;
    }
    cudaError_t e;
    if (prec == RCP_FP64)
        e = rcpk::launch_solve<double>(n, nrhs, (const double *)LA, lda, Dd, Ds, perm, X, ldx,
                                       reinterpret_cast<double *>(base), flags, status, nullptr, s);
    else
        e = rcpk::launch_solve<float>(n, nrhs, (const float *)LA, lda, Dd, Ds, perm, X, ldx,
                                      reinterpret_cast<float *>(base), flags, status, nullptr, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RCP_ECUDA;
    }
    const long long total = (long long)n * nrhs;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 1024);
    poison_on_status_kernel<<<blocks, 256, 0, s>>>(n, nrhs, X, ldx, status);
    rcpk::count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return RCP_ECUDA;
    return RCP_OK;
}
