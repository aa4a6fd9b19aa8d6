// sketch_tc.cu -- the Gaussian sketch B = Omega A of Section 3 ("draw Omega, B = Omega A" of
// Algorithm 1) on the tcgen05 tensor cores, for the FP32 factors whose trailing update runs there
// (RCP_TF32X3, RCP_F16X3).
//
// A is symmetric, so B^T = A Omega^T: one MMA tile has M = 128 columns j of B (rows of A's block
// row), N = d rounded up to 16 (the sketch rows) and runs over K = the rows k of A in chunks of
// 32.  Precision as in the trailing update: every operand x is split as x = hi + lo with
// hi = tf32(x), lo = tf32(x - hi), and hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor memory
// (about 2^-22 relative per product, an FP32 sketch).  TF32 needs no scaling, so columns of A can
// be sketched as they arrive without knowing max|A|.
//
// Work: units of (128 columns, K slice); a slice count that depends on n only keeps every column's
// sum in the same order whichever column range a launch covers (the host-buffer path sketches
// A's columns block by block as they land).  With more than one slice each unit writes its
// partial sum, and the slices are added in order afterwards.
//
// Roles per CTA (persistent over units; 13 warps):
//   warp 0, one thread: waits for a stage's operands, issues 4 K-steps x 3 tcgen05.mma
//     (kind::tf32, M = 128, N = np, K = 8) into one of two tensor-memory accumulators, commits
//     the stage back to the loaders and, after a unit's last chunk, the accumulator to the
//     epilogue;
//   warps 1-8: load the chunk's 128 x 32 block of A from global memory (a chunk ahead, in
//     registers), split it, store it into the stage's two swizzled K-major tiles (A_hi, A_lo),
//     and one thread bulk-copies the chunk's pre-split Omega tiles (np x 32, hi and lo);
//   warps 9-12: drain an accumulator (tcgen05.ld 32x32b; warp w reads lane quarter w % 4) into
//     B or the unit's partial sum, then hand the accumulator back.
// Every wait is bounded (kWaitLimitNs); a role whose wait runs out sets ST_TIMEOUT and the
// abort flag, the others stop at their next wait, copies in flight are waited for (bounded),
// and the tensor memory is freed before the CTA returns.
#include <algorithm>

#include "kernels.h"
#include "tc_common.cuh"

namespace rcpk {

namespace sktc {
constexpr int TM = 128;                          // columns of B per tile (MMA M)
constexpr int KC = 32;                           // rows of A per chunk (one 128-byte TF32 row)
constexpr int STAGES = 3;
constexpr int LOAD_WARPS = 16, EPI_WARPS = 4;
constexpr int THREADS = 32 * (1 + LOAD_WARPS + EPI_WARPS);
constexpr int LOAD_THREADS = 32 * LOAD_WARPS;
constexpr int A_FLOATS = TM * KC;                // one split part of an A chunk: 16 KB
constexpr int PER = A_FLOATS / LOAD_THREADS;     // values per loader thread and chunk
static_assert(PER == 8, "loader mapping");
static_assert(EPI_WARPS == 4, "one epilogue warp per tensor-memory lane quarter");

__host__ __device__ constexpr int npad(int d) { return (d + 15) / 16 * 16; }
__host__ __device__ constexpr size_t stage_floats(int np) { return 2 * (size_t)A_FLOATS + 2 * (size_t)np * KC; }
}  // namespace sktc

// K slices of the tensor-core sketch: a function of n alone (at least 32 chunks of 32 rows per
// slice, at most 16 slices)
int sketch_tc_slices(int n) {
    const int ksteps = (n + sktc::KC - 1) / sktc::KC;
    return std::max(1, std::min(16, ksteps / 32));
}

size_t sketch_tc_omega_floats(int n, int d) {
    const size_t nkc = ((size_t)n + sktc::KC - 1) / sktc::KC;
    return 2 * nkc * (size_t)sktc::npad(d) * sktc::KC;
}

size_t sketch_tc_scratch_floats(int n, int d) {
    const int S = sketch_tc_slices(n);
    return S > 1 ? (size_t)S * d * n : 0;
}

// Omega (d x n, ld d) as K-major swizzled tiles of np rows x 32 K values, TF32 hi and lo parts:
// tile (c, q) at (2 c + q) np 32 floats; rows r >= d and columns k >= n are zero.  With st
// (the q = b block update), the matrix is Y = B_blk L11^{-T} (d x nb) of the panel just done,
// nb = kend - k0 read from the device state.
__global__ void omega_split_kernel(int n, int d, int np, const float *__restrict__ om, float *__restrict__ out,
                                   const FactorState *st) {
    if (st) {
        const int nb = st->kend - st->k0;
        if (nb <= 0 || st->kend >= n) return;
        n = nb;
    }
    const int nkc = (n + sktc::KC - 1) / sktc::KC;
    for (int c = blockIdx.x; c < nkc; c += gridDim.x) {
        float *hi = out + (size_t)(2 * c) * np * sktc::KC, *lo = hi + (size_t)np * sktc::KC;
        for (int e = threadIdx.x; e < np * sktc::KC; e += blockDim.x) {
            const int r = e % np, kk = e / np;   // r fastest: reads along Omega's columns
            const int k = c * sktc::KC + kk;
            const float v = (r < d && k < n) ? om[(size_t)r + (size_t)k * d] : 0.f;
            const float h = tc::tf32_rna(v);
            const int o = tc::swz(r, kk);
            hi[o] = h;
            lo[o] = tc::tf32_rna(v - h);
        }
    }
}

struct SkUnit {
    int j0, kb, ke, sl;
};

__device__ __forceinline__ SkUnit sk_unit(int lu, int Jb, int S, int ksteps, int c0) {
    const int u = blockIdx.x + lu * gridDim.x;
    SkUnit x;
    x.sl = u / Jb;
    x.j0 = c0 + (u % Jb) * sktc::TM;
    x.kb = (int)((long long)ksteps * x.sl / S);
    x.ke = (int)((long long)ksteps * (x.sl + 1) / S);
    return x;
}

// Loader mapping of element u (0..7) of loader warp lw (0..15) to (m, kk) = (column j0 + m, row
// k0 + kk) of a chunk.  Above the diagonal block (k < j everywhere) A(k, j) is stored at j + k lda
// and the lanes run along j; elsewhere the lanes run along k (stored at k + j lda below the
// diagonal, mixed on it).
__device__ __forceinline__ void sk_map(bool above, int lw, int lane, int u, int *m, int *kk) {
    if (above) {
        *m = lane + 32 * (u & 3);
        *kk = lw + 16 * (u >> 2);
    } else {
        *m = lw + 16 * u;
        *kk = lane;
    }
}

// UPD = false: the sketch, columns c0 .. c1-1 of B (or of the slice partials).  UPD = true: the
// q = b block sketch update B(:, k1:n) -= Y L21^T, i.e. B^T(j, :) -= sum_c L(j, k0 + c) Y(:, c)^T
// for the rows j >= k1 of the panel's multipliers (A = Lc, position order, ld n; K = the panel's
// nb columns), its geometry read from the device state, B updated in place.
template <bool UPD>
__global__ void __launch_bounds__(sktc::THREADS, 1)
sketch_tc_kernel(int n, int d, int np, const float *__restrict__ A, int lda, const float *__restrict__ omt,
                 float *__restrict__ out, int S, int Jb, int ksteps, int c0, int c1, int *status,
                 const FactorState *st) {
    using namespace sktc;
    int kmax = n;   // K extent (rows of A, or the panel's columns)
    if (UPD) {
        if (ldcg(status) != 0) return;
        const int k0 = st->k0, k1 = st->kend;
        if (k1 - k0 <= 0 || k1 >= n) return;
        kmax = k1 - k0;
        c0 = k1;
        c1 = n;
        S = 1;
        ksteps = (kmax + KC - 1) / KC;
        Jb = (n - k1 + TM - 1) / TM;
    }
    extern __shared__ __align__(1024) unsigned char sk_smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES];   // the stage's A parts stored (one arrival per loader warp)
    __shared__ __align__(8) uint64_t om_bar[STAGES];     // its Omega parts landed (transaction count)
    __shared__ __align__(8) uint64_t free_bar[STAGES];   // the MMAs reading it completed (tcgen05.commit)
    __shared__ __align__(8) uint64_t accf[2];            // accumulator holds a finished unit
    __shared__ __align__(8) uint64_t acce[2];            // the epilogue has read it
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int units = Jb * S;
    if ((int)blockIdx.x >= units) return;
    const int nunits = (units - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    float *base = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(sk_smem_raw) + 1023) & ~(uintptr_t)1023);
    const size_t sf = stage_floats(np);
    const uint32_t om_part_bytes = (uint32_t)np * KC * 4u;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full_bar[s], LOAD_WARPS);
            tc::mbar_init(&om_bar[s], 1);
            tc::mbar_init(&free_bar[s], 1);
        }
        for (int a = 0; a < 2; ++a) { tc::mbar_init(&accf[a], 1); tc::mbar_init(&acce[a], EPI_WARPS); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" :: "r"(tc::smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *abort_flag = &s_abort;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = tc::idesc_tf32(TM, np);
            uint32_t full_ph = 0, om_ph = 0, acce_ph = 0;
            int uses[STAGES] = {0, 0, 0};
            int g = 0;
            bool ok = true;
            for (int lu = 0; lu < nunits && ok; ++lu) {
                const SkUnit x = sk_unit(lu, Jb, S, ksteps, c0);
                const int a = lu & 1;
                const uint32_t dacc = tmem + (uint32_t)(a * TM);
                if (lu >= 2) {
                    if (!tc::mbar_wait(&acce[a], (acce_ph >> a) & 1u)) { ok = false; break; }
                    acce_ph ^= 1u << a;
                    tc::tc_fence_after();
                }
                for (int c = x.kb; c < x.ke; ++c, ++g) {
                    const int s = g % STAGES;
                    if (*abort_flag || !tc::mbar_wait(&om_bar[s], (om_ph >> s) & 1u) ||
                        !tc::mbar_wait(&full_bar[s], (full_ph >> s) & 1u)) {
                        ok = false;
                        break;
                    }
                    om_ph ^= 1u << s;
                    full_ph ^= 1u << s;
                    tc::tc_fence_after();
                    const float *st = base + (size_t)s * sf;
                    const uint32_t a_hi = tc::smem_u32(st), a_lo = tc::smem_u32(st + A_FLOATS);
                    const uint32_t o_hi = tc::smem_u32(st + 2 * A_FLOATS), o_lo = tc::smem_u32(st + 2 * A_FLOATS + np * KC);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t off = kk * 32;   // one K-step of 8 TF32 values = 32 bytes along the row
                        tc::mma_tf32(dacc, tc::sdesc_k128(a_hi + off), tc::sdesc_k128(o_hi + off), idesc,
                                     (c > x.kb || kk > 0) ? 1u : 0u);
                        tc::mma_tf32(dacc, tc::sdesc_k128(a_hi + off), tc::sdesc_k128(o_lo + off), idesc, 1u);
                        tc::mma_tf32(dacc, tc::sdesc_k128(a_lo + off), tc::sdesc_k128(o_hi + off), idesc, 1u);
                    }
                    tc::mma_commit(&free_bar[s]);
                    ++uses[s];
                }
                if (!ok) break;
                tc::mma_commit(&accf[a]);
            }
            if (!ok) {
                *abort_flag = 1;
                atomicOr(status, ST_TIMEOUT);
            }
            // the MMAs of the last commit of every stage complete before the tensor memory is freed
            for (int s = 0; s < STAGES; ++s)
                if (uses[s] > 0) tc::mbar_wait(&free_bar[s], (uint32_t)((uses[s] - 1) & 1));
        }
    } else if (warp <= LOAD_WARPS) {
        // ---------------- loaders ----------------
        const int lt = tid - 32, lw = lt >> 5;
        uint32_t free_ph = 0;
        int issued[STAGES] = {0, 0, 0};   // Omega copies issued per stage (thread lt == 0)
        float bufa[PER], bufb[PER];
        auto load_chunk = [&](float (&v)[PER], int j0, int c) {
            const int k0 = c * KC;
            const bool above = UPD || k0 + KC <= j0;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                int m, kk;
                sk_map(above, lw, lane, u, &m, &kk);
                const int j = j0 + m, k = k0 + kk;
                float x = 0.f;
                if (UPD) {
                    if (k < kmax && j < c1) x = A[(size_t)j + (size_t)k * lda];   // L(j, k0 + k)
                } else if (k < n && j < c1) {
                    x = k >= j ? A[(size_t)k + (size_t)j * lda] : A[(size_t)j + (size_t)k * lda];
                }
                v[u] = x;
            }
        };
        // two cursors over this CTA's (unit, chunk) sequence: the loads run two chunks ahead of
        // the stores, alternating between two register buffers
        struct Cursor {
            int lu, c;
            SkUnit x;
            bool live;
        };
        auto first = [&]() { Cursor q{0, 0, sk_unit(0, Jb, S, ksteps, c0), nunits > 0}; q.c = q.x.kb; return q; };
        auto step = [&](Cursor &q) {
            if (++q.c < q.x.ke) return;
            if (++q.lu < nunits) {
                q.x = sk_unit(q.lu, Jb, S, ksteps, c0);
                q.c = q.x.kb;
            } else {
                q.live = false;
            }
        };
        Cursor ld = first(), pr = first();
        // store the chunk of buffer v at the stage of chunk g (false: a wait ran out)
        auto store_chunk = [&](const float (&v)[PER], int g) -> bool {
            const int s = g % STAGES;
            if (g >= STAGES) {
                const bool ok = !*abort_flag && tc::mbar_wait(&free_bar[s], (free_ph >> s) & 1u);
                if (!ok) {
                    *abort_flag = 1;
                    atomicOr(status, ST_TIMEOUT);
                    return false;
                }
                free_ph ^= 1u << s;
            }
            float *st = base + (size_t)s * sf;
            if (lt == 0) {
                const float *src = omt + (size_t)(2 * pr.c) * np * KC;
                const uint64_t keep = tc::policy_evict_last();
                tc::mbar_expect_tx(&om_bar[s], 2 * om_part_bytes);
                tc::bulk_g2s(st + 2 * A_FLOATS, src, om_part_bytes, &om_bar[s], keep);
                tc::bulk_g2s(st + 2 * A_FLOATS + np * KC, src + (size_t)np * KC, om_part_bytes, &om_bar[s], keep);
                ++issued[s];
            }
            const bool above = UPD || pr.c * KC + KC <= pr.x.j0;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                int m, kk;
                sk_map(above, lw, lane, u, &m, &kk);
                const int o = tc::swz(m, kk);
                const float h = tc::tf32_rna(v[u]);
                st[o] = h;
                st[A_FLOATS + o] = tc::tf32_rna(v[u] - h);
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&full_bar[s]);
            step(pr);
            return true;
        };
        bool fa = ld.live, fb = false;
        if (fa) { load_chunk(bufa, ld.x.j0, ld.c); step(ld); }
        fb = ld.live;
        if (fb) { load_chunk(bufb, ld.x.j0, ld.c); step(ld); }
        for (int g = 0; fa; g += 2) {
            if (!store_chunk(bufa, g)) break;
            fa = ld.live;
            if (fa) { load_chunk(bufa, ld.x.j0, ld.c); step(ld); }
            if (!fb) break;
            if (!store_chunk(bufb, g + 1)) break;
            fb = ld.live;
            if (fb) { load_chunk(bufb, ld.x.j0, ld.c); step(ld); }
        }
        // no bulk copy may still be writing this CTA's shared memory when it returns
        if (lt == 0)
            for (int s = 0; s < STAGES; ++s)
                if (issued[s] > 0) tc::mbar_wait(&om_bar[s], (uint32_t)((issued[s] - 1) & 1));
    } else {
        // ---------------- epilogue: lane quarter q, column j0 + 32 q + lane ----------------
        const int q = warp & 3;
        uint32_t accf_ph = 0;
        for (int lu = 0; lu < nunits; ++lu) {
            const SkUnit x = sk_unit(lu, Jb, S, ksteps, c0);
            const int a = lu & 1;
            if (*abort_flag) break;
            if (!tc::mbar_wait(&accf[a], (accf_ph >> a) & 1u)) {
                *abort_flag = 1;
                atomicOr(status, ST_TIMEOUT);
                break;
            }
            accf_ph ^= 1u << a;
            tc::tc_fence_after();
            const int j = x.j0 + q * 32 + lane;
            float *dst = UPD ? out + (size_t)j * d : out + (size_t)x.sl * d * (c1 - c0) + (size_t)(j - c0) * d;
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * TM);
            for (int cb = 0; cb < np; cb += 16) {
                uint32_t r[16];
                tc::tmem_ld16(taddr + (uint32_t)cb, r);
                tc::tmem_wait_ld();
                if (j < c1) {
#pragma unroll
                    for (int t = 0; t < 16; ++t)
                        if (cb + t < d) {
                            if (UPD) dst[cb + t] -= __uint_as_float(r[t]);
                            else dst[cb + t] = __uint_as_float(r[t]);
                        }
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[a]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem) : "memory");
}

// SM count; the dynamic shared-memory limit of both kernel variants is raised once (for np = 128)
static int sk_setup() {
    static int sms = 0;
    if (!sms) {
        int dev = 0, m = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
        const int want = (int)(sktc::STAGES * sktc::stage_floats(128) * sizeof(float) + 1024);
        if (cudaFuncSetAttribute(sketch_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, want) !=
                cudaSuccess ||
            cudaFuncSetAttribute(sketch_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, want) !=
                cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        sms = m;
    }
    return sms;
}

cudaError_t launch_omega_split(int n, int d, const float *om, float *omt, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (d < 1 || d > 128) return cudaErrorInvalidValue;
    const int nkc = (n + sktc::KC - 1) / sktc::KC;
    omega_split_kernel<<<std::min(nkc, 4096), 256, 0, s>>>(n, d, sktc::npad(d), om, omt, nullptr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sketch_tc(int n, int d, const float *A, int lda, const float *omt, float *B, float *part,
                             size_t part_floats, int c0, int c1, int *status, cudaStream_t s) {
    using namespace sktc;
    if (n == 0 || c1 <= c0) return cudaSuccess;
    if (d < 1 || d > 128 || c0 < 0 || c1 > n || !status) return cudaErrorInvalidValue;
    const int np = npad(d);
    const size_t smem = STAGES * stage_floats(np) * sizeof(float) + 1024;
    const int sms = sk_setup();
    if (sms <= 0) return cudaErrorInvalidValue;
    const int nc = c1 - c0;
    const int Jb = (nc + TM - 1) / TM, ksteps = (n + KC - 1) / KC;
    const int S = sketch_tc_slices(n);
    if (S > 1 && (!part || part_floats < (size_t)S * d * nc)) return cudaErrorInvalidValue;
    float *dst = S > 1 ? part : B + (size_t)c0 * d;
    const int grid = std::min(Jb * S, sms);
    sketch_tc_kernel<false><<<grid, THREADS, smem, s>>>(n, d, np, A, lda, omt, dst, S, Jb, ksteps, c0, c1, status,
                                                        nullptr);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (S > 1) return launch_sketch_reduce((size_t)d * nc, S, part, B + (size_t)c0 * d, s);
    return cudaSuccess;
}

size_t block_update_tc_floats(int bw, int d) {
    const size_t nkc = ((size_t)bw + sktc::KC - 1) / sktc::KC;
    return 2 * nkc * (size_t)sktc::npad(d) * sktc::KC;
}

cudaError_t launch_block_sketch_update_tc(const FactorWork<float> &w, float *ytmp, float *ytiles, cudaStream_t s) {
    using namespace sktc;
    if (w.d < 1 || w.d > 128) return cudaErrorInvalidValue;
    cudaError_t e = launch_bsk_y<float>(w, ytmp, s);   // Y = B(:, k0:k1) L11^{-T} (CUDA cores, small)
    if (e != cudaSuccess) return e;
    const int np = npad(w.d);
    const int nkc = (w.bw + KC - 1) / KC;
    omega_split_kernel<<<nkc, 256, 0, s>>>(w.n, w.d, np, ytmp, ytiles, w.st);
    count_launches(1);
    const int sms = sk_setup();
    if (sms <= 0) return cudaErrorInvalidValue;
    const int grid = std::min((w.n + TM - 1) / TM, sms);
    const size_t smem = STAGES * stage_floats(np) * sizeof(float) + 1024;
    sketch_tc_kernel<true><<<grid, THREADS, smem, s>>>(w.n, w.d, np, w.Lc, w.n, ytiles, w.B, 1, 1, 1, 0, 0, w.status,
                                                       w.st);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rcpk
