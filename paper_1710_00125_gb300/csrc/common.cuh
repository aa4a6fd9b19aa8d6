// common.cuh -- device helpers shared by the RCP kernels: status bits, bounded grid
// barrier, L2-coherent loads and stores, and the per-factorization device state.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rcpk {

// Host-side count of kernel launches issued by this library (for benchmark reporting).
void count_launches(long long k);

// Bits of the device status word.
enum : int {
    ST_TIMEOUT = 1,      // a bounded wait ran out
    ST_NONFINITE = 2,    // NaN/Inf met in a pivot, a multiplier or a norm
    ST_INTERNAL = 4      // an internal size check failed (the kernel skipped its work)
};

// Upper bound on a single device-side wait (nanoseconds of %globaltimer).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s

// Programmatic dependent launch between the kernels of one panel (gather, scatter, panel store,
// panel record, tile preparation, trailing update): each of them is launched with the stream's
// programmatic serialization allowed, and waits for its predecessor's completion (and memory) at
// its first instruction, so only the launch itself overlaps the predecessor's last wave.  A
// predecessor lets its successor's launch begin once all of its CTAs are running.  Both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Device state of one factorization, kept in handle workspace.
struct FactorState {
    int next;        // first column of the next panel
    int k0;          // first column of the current panel
    int kend;        // one past its last column
    int info;        // 1 + first zero pivot, 0 if none
    int n2x2;        // 2x2 blocks so far
    int n_moved;     // entries in the moved list of the current panel
    int guard_req;   // Algorithm 2, set by the panel: 1 recompute the sketch at guard_k, 2 stop there
    int guard_k;     // position where the panel stopped for the safeguard
    double beta2;           // ||B^(1)||_{1,2}^2 (largest initial sketch column norm^2)
    double min_ratio;       // min over steps of ||B(:, pi)|| / sqrt(beta2)
    unsigned long long maxD_bits;   // max |D_ij| as ordered bits of a non-negative double
    unsigned long long maxL_bits;   // max |L_ij|
    unsigned long long maxA_bits;   // max |A_ij| of the input
    unsigned long long tcW_bits;    // max |W| over the current panel's trailing rows (FP16 split
    unsigned long long tcL_bits;    //   update) and max |L21|; ordered bits of non-negative doubles
    int nresk;              // Algorithm 2: sketch recomputations so far
    int rank;               // Algorithm 2: columns eliminated before a rank-deficiency stop (n if none)
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_s32(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Loads/stores of data exchanged between CTAs inside one kernel: cached in L2 only.
template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void stcg(T *p, T v) { __stcg(p, v); }

// Grid-wide barrier for a cooperative launch.  `bar` counts arrivals; the barrier with
// sequence number `seq` (1, 2, ...) completes when bar >= base + seq * nblocks.  The wait is
// bounded by limit_ns (kWaitLimitNs unless a caller asks for less); on expiry ST_TIMEOUT is
// set and false is returned to every thread of the CTA.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned target, int *status,
                                             unsigned long long limit_ns = kWaitLimitNs) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        // the CTA's writes are ordered before this release by the __syncthreads above
        red_release_add_u32(bar, 1u);
        int ok = 1;
        if (ld_acquire_u32(bar) < target) {
            unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_u32(bar) < target) {
                if ((++spins & 255u) == 0 && global_ns() - t0 > limit_ns) {
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

// The same barrier in two halves, so that a CTA can work between its arrival and its wait:
// grid_arrive orders the CTA's earlier writes before the arrival (every thread must call it);
// grid_wait returns the bounded wait's outcome to every thread.
__device__ __forceinline__ void grid_arrive(unsigned *bar) {
    __syncthreads();
    if (threadIdx.x == 0) red_release_add_u32(bar, 1u);
}

__device__ __forceinline__ bool grid_wait(unsigned *bar, unsigned target, int *status) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_u32(bar) < target) {
            unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_u32(bar) < target) {
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

// Base of the arrival counter at kernel entry: every launch completes all its barriers, so
// the counter is a multiple of nblocks when no CTA of this launch has arrived yet, and at
// most nblocks-1 arrivals of this launch can precede any CTA's read.
__device__ __forceinline__ unsigned barrier_base(const unsigned *bar, unsigned nblocks) {
    unsigned v = ld_acquire_u32(bar);
    return (v / nblocks) * nblocks;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    if (v > 0.0 || v == 0.0) atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }


// ---- packed 64-bit argmax keys (FP32 values) exchanged between the CTAs of a grid ----------
// FP32 argmax key: larger key = larger value, then smaller position.  Needs n <= 65535.
__device__ __forceinline__ unsigned long long make_key(float v, int lpos, int phys) {
    return ((unsigned long long)__float_as_uint(v) << 32) | ((unsigned long long)(0xFFFFu - (unsigned)lpos) << 16) |
           (unsigned long long)(unsigned)phys;
}

__device__ __forceinline__ void red_max_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Keys are read right after the grid barrier, whose acquire already orders these loads after
// every CTA's red.max; a relaxed load suffices and lets independent key loads overlap.
__device__ __forceinline__ unsigned long long ld_key(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Ring of key slots indexed by the grid-barrier generation; the slot of generation g + KEY_RING/2
// is cleared (by one CTA) after the key of generation g is read, so a slot is zero when reused.
// Each slot has a 128-byte line of its own (KEY_STRIDE words), so that the clearing store and
// the red.max of the current generation do not meet on one line.
constexpr int KEY_RING = 16;
constexpr int KEY_STRIDE = 16;

__device__ __forceinline__ unsigned long long *key_slot(unsigned long long *ring, unsigned g) {
    return ring + (size_t)(g % KEY_RING) * KEY_STRIDE;
}

// Maximum of a packed key over the warp (the result in every lane): redux.sync on the high
// words, then on the low words among the lanes holding the maximal high word.
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const unsigned m = __reduce_max_sync(0xffffffffu, hi);
    const unsigned l = __reduce_max_sync(0xffffffffu, hi == m ? lo : 0u);
    return ((unsigned long long)m << 32) | l;
}

}  // namespace rcpk
