// trailing_tc.cu -- the deferred trailing update of Algorithm 1, A22 -= W L21^T (lower triangle),
// on the 5th-generation tensor cores (tcgen05, accumulators in tensor memory) for FP32 factors.
//
// Precision: W and L21 are FP32.  With plain TF32 inputs (10-bit mantissa) the update error
// is ~1e-3 relative, too large for FP64 refinement to converge at condition numbers of 1e4.
// Each operand is split as x = hi + lo with hi = tf32(x), lo = tf32(x - hi), and three products
// hi*hi + hi*lo + lo*hi are accumulated in FP32 (the dropped lo*lo term is ~2^-22 relative).
// The FP16 variant splits the same way in FP16, whose 11 significant bits equal TF32's: before
// the split W is multiplied by 2^sw and L21 by 2^sl, the powers of two that put the panel's
// max |W| and max |L21| (reduced by the panel kernel as it publishes them) in [2^14, 2^15),
// below the FP16 maximum; the
// epilogue multiplies the accumulator by 2^-sw 2^-sl (exact).  An entry keeps the full 22 bits
// of its two parts while its low part is an FP16 normal, i.e. down to 2^-18 of the panel maximum;
// the parts of smaller entries lose bits only far below the update's normwise FP32 error.  The
// FP16 products run at twice the TF32 rate, and a 16 KB operand tile carries K = 64 instead of 32,
// which halves the operand traffic per product.
//
// Data path per panel:
//   prep kernel: rows kend..n of W (Wbuf) and of L21 (the panel columns of A) are rounded to
//     hi/lo and written as K-major 128-row tiles of 128-byte rows (32 TF32 or 64 FP16 columns),
//     in the exact shared-memory image of
//     the 128-byte swizzle (16 KB per tile, contiguous), one tile per (row block, K chunk).
//   MMA kernel: persistent CTAs walk the 128 x 256 super-tiles (row block I, column tiles J0 and
//     J0 + 1, I >= J0) of the trailing lower triangle.  Per K chunk one thread issues six 16 KB
//     bulk copies (W_hi, W_lo of row block I; L_hi, L_lo of column tiles J0 and J0 + 1) into a
//     2-stage ring of 96 KB guarded by mbarriers, then 4 K-steps x 3 tcgen05.mma (M = 128,
//     N = 256, K = 8 in TF32, 16 in FP16) into one of two 256-column TMEM accumulators, and
//     commits the stage back to its "free" barrier.  After the last chunk the accumulator is
//     drained by sixteen warps (tcgen05.ld 32x32b: TMEM lane quarter w % 4, 64 of the 256 columns
//     each) and subtracted from A in place, while the MMAs of the next super-tile fill the other.
// Every wait is bounded (kWaitLimitNs); on expiry the status word is set, the CTA stops
// issuing work, waits for its issued copies and MMAs (bounded), frees its tensor memory and
// returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"
#include "tc_common.cuh"

namespace rcpk {

namespace tc {

constexpr int TM = 128;              // tile rows (M); a super-tile has NT 128-column tiles (N = 128 NT)
constexpr int TILE_FLOATS = 4096;    // one 128 x 128-byte tile = 16 KB
constexpr int NT = 2;                // 128 x 256 super-tiles: the W tile of a chunk serves two L tiles
constexpr int STAGES = NT == 1 ? 3 : 2;
constexpr uint32_t STAGE_BYTES = (2u + 2u * NT) * TILE_FLOATS * 4u;   // W_hi, W_lo, L_hi x NT, L_lo x NT
// K chunk: one 128-byte swizzle row, 32 TF32 or 64 FP16 values
template <bool F16> constexpr int KC = F16 ? 64 : 32;

// Scale exponent for the FP16 split: the largest e with bound * 2^e < 2^15 (0 for a zero or
// non-finite bound), from the bits of a non-negative double; clamped to the FP32 range.
__device__ __forceinline__ int f16_scale_exp(unsigned long long bits) {
    const int ef = (int)((bits >> 52) & 0x7FFu);   // biased exponent: bound < 2^(ef - 1022)
    if (bits == 0ull || ef == 0x7FF) return 0;
    const int e = ef == 0 ? -1022 : ef - 1022;
    const int s = 15 - e;
    return s < -126 ? -126 : (s > 126 ? 126 : s);
}

// Instruction descriptors: D = F32, A = B = TF32 (kind::tf32) or F16 (kind::f16), both
// K-major, M = 128, N = 128 NT.
constexpr uint32_t IDESC_TF32 =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)((TM * NT) >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t IDESC_F16 =
    (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)((TM * NT) >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

template <bool F16>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    if (F16)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(IDESC_F16), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(IDESC_TF32), "r"(accumulate)
            : "memory");
}

}  // namespace tc

// ------------------------------------------------------------------------------------------
// prep: hi/lo split of W(kend:n, 0:K) and L21 = A(kend:n, k0:kend) into swizzled tiles.
// Tile (R, c) of an operand starts at (R * nkc + c) * TILE_FLOATS; rows past n and columns past
// K are zero.  Layout of the operand buffer: [W_hi | W_lo | L_hi | L_lo], each nrb * nkc tiles.
// ------------------------------------------------------------------------------------------
// One CTA per (row block R, K chunk c): coalesced column reads of W and L21, the hi/lo split,
// the swizzle in shared memory, then contiguous 16-byte stores of the four 16 KB tiles.
template <bool F16>
__global__ void __launch_bounds__(256) tc_prep_kernel(FactorWork<float> w, float *ops, int nrb_cap, int nkc_cap) {
    constexpr int KC = tc::KC<F16>;
    __shared__ __align__(16) float t2[2][tc::TILE_FLOATS];   // hi, lo images of one operand tile (32 KB)
    pdl_wait();
    pdl_release();
    if (ldcg(w.status) != 0) return;
    const int n = w.n, lda = w.lda, k0 = w.st->k0, kend = w.st->kend;
    const int K = kend - k0, N = n - kend;
    if (K <= 0 || N <= 0) return;
    const int nrb = (N + tc::TM - 1) / tc::TM, nkc = (K + KC - 1) / KC;
    if (nrb > nrb_cap || nkc > nkc_cap) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(w.status, ST_INTERNAL);
        return;
    }
    float scale[2] = {1.f, 1.f};   // FP16: 2^sw for W, 2^sl for L21
    if (F16) {
        scale[0] = ldexpf(1.f, tc::f16_scale_exp(ldcg(&w.st->tcW_bits)));
        scale[1] = ldexpf(1.f, tc::f16_scale_exp(ldcg(&w.st->tcL_bits)));
    }
    const size_t per = (size_t)nrb_cap * nkc_cap * tc::TILE_FLOATS;
    const uint64_t keep = tc::policy_evict_last();
    for (int tile = blockIdx.x; tile < nrb * nkc; tile += gridDim.x) {
        const int R = tile / nkc, c = tile % nkc;
        const size_t toff = ((size_t)R * nkc + c) * tc::TILE_FLOATS;
        for (int op = 0; op < 2; ++op) {   // 0: W rows, 1: L21 rows
            // all of this thread's loads first (the reads miss L2: many in flight), then the split
            // element u of this thread: row m = tid % 128, K index kk = tid / 128 + 2 u
            constexpr int PER = tc::TM * KC / 256;
            static_assert(tc::TM * KC % 256 == 0 && 256 % tc::TM == 0, "elements per thread");
            const int m = threadIdx.x % tc::TM, kk0 = threadIdx.x / tc::TM;
            const int p = kend + R * tc::TM + m;
            const int kleft = p < n ? K - (c * KC + kk0) : 0;   // elements u < (kleft + 1) / 2 exist
            const size_t ld = op == 0 ? (size_t)n : (size_t)lda;
            const float *src = (op == 0 ? w.Wbuf + (size_t)(c * KC + kk0) * n : w.A + (size_t)(k0 + c * KC + kk0) * lda) +
                               (p < n ? p : 0);
            float v[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) v[u] = 2 * u < kleft ? src[(size_t)(2 * u) * ld] : 0.f;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int kk = kk0 + 2 * u;
                if (F16) {
                    const float xs = v[u] * scale[op];
                    const __half h = __float2half_rn(xs);
                    const int o = tc::swz16(m, kk);
                    reinterpret_cast<__half *>(t2[0])[o] = h;
                    reinterpret_cast<__half *>(t2[1])[o] = __float2half_rn(xs - __half2float(h));
                } else {
                    const float h = tc::tf32_rna(v[u]);
                    const int o = tc::swz(m, kk);
                    t2[0][o] = h;
                    t2[1][o] = tc::tf32_rna(v[u] - h);
                }
            }
            __syncthreads();
            for (int q = 0; q < 2; ++q) {
                float4 *dst = reinterpret_cast<float4 *>(ops + (size_t)(2 * op + q) * per + toff);
                const float4 *src = reinterpret_cast<const float4 *>(t2[q]);
                for (int v = threadIdx.x; v < tc::TILE_FLOATS / 4; v += blockDim.x) tc::st_keep_v4(dst + v, src[v], keep);
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------------------------
// tcgen05 MMA kernel, warp-specialized.  Warp 0 (one elected thread) streams operand chunks
// through the stage ring and issues the MMAs of each super-tile into one of two 256-column TMEM
// accumulators; warps 1..16 drain the other accumulator (tcgen05.ld: lane quarter w % 4, a
// 64-column quarter each) and update A, so the epilogue of super-tile t overlaps the MMAs of t + 1.
// Each epilogue warp reads its 32 x 64 block of A in four 16-column chunks, two chunks ahead:
// the first two are loaded before it waits for the accumulator, so the HBM latency of the
// read-modify-write stays behind the MMAs.  Sixteen epilogue warps (not eight) keep twice the
// bytes of A in flight per SM; 17 warps leave 96 registers per thread, which two chunks fit.
//   full[s]  : operands of the chunk in stage s arrived (bulk-copy transaction count)
//   free[s]  : the MMAs reading stage s completed (tcgen05.commit)
//   accf[a]  : accumulator a holds a finished tile (tcgen05.commit)
//   acce[a]  : the epilogue has read accumulator a (one arrival per epilogue warp)
// ------------------------------------------------------------------------------------------
constexpr int TC_EPI_WARPS = 16;
constexpr int TC_EPI_COLS = tc::TM * tc::NT * 4 / TC_EPI_WARPS;   // columns per epilogue warp
constexpr int TC_THREADS = 32 * (1 + TC_EPI_WARPS);


// Tile order with NT = 1: diagonal by diagonal (delta = I - J = 0, 1, ...; J ascending within a
// diagonal).  Diagonal delta holds nrb - delta tiles and starts at C(delta) = delta (2 nrb + 1 -
// delta) / 2.
__device__ __forceinline__ void tile_ij(long long tile, int nrb, int *I, int *J) {
    // FP32 estimate of the root of delta^2 - (2 nrb + 1) delta + 2 tile = 0, corrected in integers
    // (no FP64 on this part's slow FP64 pipe)
    const float b = 2.f * (float)nrb + 1.f;
    const float disc = fmaxf(b * b - 8.f * (float)tile, 0.f);
    int dl = (int)((b - sqrtf(disc)) * 0.5f);
    dl = dl < 0 ? 0 : (dl > nrb - 1 ? nrb - 1 : dl);
    auto start = [&](long long x) { return x * (2LL * nrb + 1 - x) / 2; };
    while (dl > 0 && start(dl) > tile) --dl;
    while (dl + 1 < nrb && start(dl + 1) <= tile) ++dl;
    *J = (int)(tile - start(dl));
    *I = *J + dl;
}

// Super-tiles of NT = 2 column tiles: row block I holds floor(I/2) + 1 of them, column tiles
// (2 J2, 2 J2 + 1), J2 = 0..floor(I/2) (on even I the last one's second tile lies above the
// diagonal: computed, never stored).  Rows come in pairs (2P, 2P+1) of P + 1 super-tiles each;
// P(P + 1) super-tiles precede pair P.  Returns the row block and the first column tile.
__device__ __forceinline__ void supertile_ij(long long t, int nrb, int *I, int *J0) {
    if (tc::NT == 1) {
        tile_ij(t, nrb, I, J0);
        return;
    }
    int P = (int)((sqrtf(4.f * (float)t + 1.f) - 1.f) * 0.5f);
    if (P < 0) P = 0;
    while (P > 0 && (long long)P * (P + 1) > t) --P;
    while ((long long)(P + 1) * (P + 2) <= t) ++P;
    const int u = (int)(t - (long long)P * (P + 1));
    const int second = u >= P + 1 ? 1 : 0;
    *I = 2 * P + second;
    *J0 = 2 * (u - second * (P + 1));
}

__host__ __device__ __forceinline__ long long supertile_count(long long nrb) {
    if (tc::NT == 1) return nrb * (nrb + 1) / 2;
    const long long m = nrb / 2;
    return (nrb & 1) ? (m + 1) * (m + 1) : m * (m + 1);
}

template <bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_trailing_kernel(FactorWork<float> w, const float *ops, int nrb_cap,
                                                                    int nkc_cap) {
    constexpr int KC = tc::KC<F16>;
    constexpr int NT = tc::NT, STAGES = tc::STAGES;
    constexpr int SN = tc::TM * NT;   // columns of a super-tile (the MMA's N)
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t free_bar[STAGES];
    __shared__ __align__(8) uint64_t accf[2];
    __shared__ __align__(8) uint64_t acce[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    pdl_wait();
    if (ldcg(w.status) != 0) return;
    const int n = w.n, lda = w.lda, k0 = w.st->k0, kend = w.st->kend;
    const int K = kend - k0, N = n - kend;
    if (K <= 0 || N <= 0) return;
    const int nrb = (N + tc::TM - 1) / tc::TM, nkc = (K + KC - 1) / KC;
    if (nrb > nrb_cap || nkc > nkc_cap) return;   // prep has flagged it
    const long long total = supertile_count(nrb);
    if ((long long)blockIdx.x >= total) return;
    const int ntiles = (int)((total - blockIdx.x + gridDim.x - 1) / gridDim.x);   // super-tiles of this CTA

    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    float *stage0 = reinterpret_cast<float *>(base);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) { tc::mbar_init(&full_bar[s], 1); tc::mbar_init(&free_bar[s], 1); }
        for (int a = 0; a < 2; ++a) { tc::mbar_init(&accf[a], 1); tc::mbar_init(&acce[a], TC_EPI_WARPS); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        // two FP32 128 x SN accumulators (2 SN <= 512 columns)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(tc::smem_u32(&s_tmem)), "r"(2 * SN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;

    const size_t per = (size_t)nrb_cap * nkc_cap * tc::TILE_FLOATS;
    const float *whi = ops, *wlo = ops + per, *lhi = ops + 2 * per, *llo = ops + 3 * per;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer + MMA issuer ----------------
            uint32_t full_ph = 0, free_ph = 0;   // phase bit per stage
            int used[STAGES] = {}, loaded[STAGES] = {};
            uint32_t acce_ph[2] = {0, 0};
            const int nchunks = ntiles * nkc;          // every chunk of every super-tile, in order
            bool ok = true;
            const uint64_t keep = tc::policy_evict_last();
            auto load = [&](int g) -> bool {
                const int s = g % STAGES;
                if (used[s]) {
                    if (!tc::mbar_wait(&free_bar[s], (free_ph >> s) & 1u)) return false;
                    free_ph ^= 1u << s;
                    used[s] = 0;
                }
                const int lt = g / nkc, c = g % nkc;
                int I, J0;
                supertile_ij(blockIdx.x + (long long)lt * gridDim.x, nrb, &I, &J0);
                const size_t ti = ((size_t)I * nkc + c) * tc::TILE_FLOATS;
                // column tiles past the last row block are not copied: their accumulator columns
                // belong to columns >= n, which the epilogue never stores
                const int nj = min(NT, nrb - J0);
                float *dst = stage0 + (size_t)s * (tc::STAGE_BYTES / 4);
                tc::mbar_expect_tx(&full_bar[s], (uint32_t)(2 + 2 * nj) * tc::TILE_FLOATS * 4u);
                tc::bulk_g2s(dst, whi + ti, tc::TILE_FLOATS * 4, &full_bar[s], keep);
                tc::bulk_g2s(dst + tc::TILE_FLOATS, wlo + ti, tc::TILE_FLOATS * 4, &full_bar[s], keep);
                for (int u = 0; u < nj; ++u) {
                    const size_t tj = ((size_t)(J0 + u) * nkc + c) * tc::TILE_FLOATS;
                    tc::bulk_g2s(dst + (2 + u) * tc::TILE_FLOATS, lhi + tj, tc::TILE_FLOATS * 4, &full_bar[s], keep);
                    tc::bulk_g2s(dst + (2 + NT + u) * tc::TILE_FLOATS, llo + tj, tc::TILE_FLOATS * 4, &full_bar[s],
                                 keep);
                }
                loaded[s] = 1;
                return true;
            };
            for (int g = 0; g < nchunks && g < STAGES && ok; ++g) ok = load(g);
            for (int g = 0; g < nchunks && ok; ++g) {
                const int lt = g / nkc, c = g % nkc, a = lt & 1;
                const uint32_t dacc = tmem + (uint32_t)(a * SN);
                if (c == 0 && lt >= 2) {
                    // accumulator a is free once the epilogue has read super-tile lt - 2
                    if (!tc::mbar_wait(&acce[a], acce_ph[a])) { ok = false; break; }
                    acce_ph[a] ^= 1u;
                    tc::tc_fence_after();
                }
                const int s = g % STAGES;
                if (!tc::mbar_wait(&full_bar[s], (full_ph >> s) & 1u)) { ok = false; break; }
                full_ph ^= 1u << s;
                loaded[s] = 0;
                tc::tc_fence_after();
                const float *st = stage0 + (size_t)s * (tc::STAGE_BYTES / 4);
                const uint32_t a_hi = tc::smem_u32(st), a_lo = tc::smem_u32(st + tc::TILE_FLOATS);
                const uint32_t b_hi = tc::smem_u32(st + 2 * tc::TILE_FLOATS);
                const uint32_t b_lo = tc::smem_u32(st + (2 + NT) * tc::TILE_FLOATS);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t off = kk * 32;   // one K-step (8 tf32 or 16 f16) = 32 bytes along the swizzled row
                    tc::mma<F16>(dacc, tc::sdesc_k128(a_hi + off), tc::sdesc_k128(b_hi + off), (c > 0 || kk > 0) ? 1u : 0u);
                    tc::mma<F16>(dacc, tc::sdesc_k128(a_hi + off), tc::sdesc_k128(b_lo + off), 1u);
                    tc::mma<F16>(dacc, tc::sdesc_k128(a_lo + off), tc::sdesc_k128(b_hi + off), 1u);
                }
                tc::mma_commit(&free_bar[s]);
                used[s] = 1;
                if (c == nkc - 1) tc::mma_commit(&accf[a]);
                // refill the stage of the previous chunk (its MMAs were queued before these)
                if (g >= 1 && g - 1 + STAGES < nchunks) ok = load(g - 1 + STAGES);
            }
            if (!ok) {
                s_abort = 1;
                atomicOr(w.status, ST_TIMEOUT);
            }
            // drain the ring before the CTA can leave
            for (int s = 0; s < STAGES; ++s) {
                if (loaded[s]) tc::mbar_wait(&full_bar[s], (full_ph >> s) & 1u);
                if (used[s]) tc::mbar_wait(&free_bar[s], (free_ph >> s) & 1u);
            }
        }
    } else {
        // ---------------- epilogue warps: lane quarter q, columns h*EC .. h*EC+EC-1 ----------------
        constexpr int EC = TC_EPI_COLS;
        static_assert(EC % 32 == 0, "pairs of 16-column chunks per epilogue warp");
        const int q = warp & 3, h = (warp - 1) >> 2;
        // FP16: the accumulator holds 2^(sw + sl) W L21^T
        float inv_w = 1.f, inv_l = 1.f;
        if (F16) {
            inv_w = ldexpf(1.f, -tc::f16_scale_exp(ldcg(&w.st->tcW_bits)));
            inv_l = ldexpf(1.f, -tc::f16_scale_exp(ldcg(&w.st->tcL_bits)));
        }
        uint32_t accf_ph[2] = {0, 0};
        float *__restrict__ A = w.A;
        const uint64_t stream = tc::policy_evict_first();   // A22 passes through L2 once per panel
        for (int lt = 0; lt < ntiles; ++lt) {
            const int a = lt & 1;
            int I, J0;
            supertile_ij(blockIdx.x + (long long)lt * gridDim.x, nrb, &I, &J0);
            const int p = kend + I * tc::TM + q * 32 + lane;
            const int q0 = kend + J0 * tc::TM + h * EC;
            // the first two 16-column chunks of the block of A this warp updates, loaded while the
            // MMAs run; every later chunk is loaded two chunks ahead of its use
            const bool rowok = p < n;
            float *blk = A + (size_t)(rowok ? p : 0) + (size_t)q0 * lda;
            float c0v[16], c1v[16];
            auto load16 = [&](float (&dst)[16], int cb) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int qq = q0 + cb + j;
                    dst[j] = (rowok && qq < n && p >= qq) ? tc::ld_stream(blk + (unsigned)((cb + j) * lda), stream) : 0.f;
                }
            };
            auto finish16 = [&](float (&src)[16], int cb, uint32_t taddr) {
                uint32_t r[16];
                tc::tmem_ld16(taddr + cb, r);
                tc::tmem_wait_ld();
                if (rowok) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int qq = q0 + cb + j;
                        if (qq < n && p >= qq) {
                            const float u = F16 ? (__uint_as_float(r[j]) * inv_w) * inv_l : __uint_as_float(r[j]);
                            tc::st_stream(blk + (unsigned)((cb + j) * lda), src[j] - u, stream);
                        }
                    }
                }
            };
            load16(c0v, 0);
            load16(c1v, 16);
            bool ok = tc::mbar_wait(&accf[a], accf_ph[a]);
            accf_ph[a] ^= 1u;
            if (!ok || *(volatile int *)&s_abort) {
                if (!ok) atomicOr(w.status, ST_TIMEOUT);
                break;
            }
            tc::tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * SN + h * EC);
#pragma unroll 1
            for (int cb = 0; cb < EC; cb += 32) {
                finish16(c0v, cb, taddr);
                if (cb + 32 < EC) load16(c0v, cb + 32);
                finish16(c1v, cb + 16, taddr);
                if (cb + 48 < EC) load16(c1v, cb + 48);
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[a]);   // the accumulator may be reused
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * SN) : "memory");
}

size_t tc_ops_floats(int n, int bmax) {
    // sized for the TF32 chunks (K = 32), which need at least as many tiles as the FP16 ones
    const size_t nrb = ((size_t)n + tc::TM - 1) / tc::TM;
    const size_t nkc = ((size_t)bmax + 1 + tc::KC<false> - 1) / tc::KC<false>;
    return 4 * nrb * nkc * tc::TILE_FLOATS;
}

template <bool F16>
static cudaError_t launch_trailing_tc_fmt(const FactorWork<float> &w, float *ops, int kmin, cudaStream_t s) {
    constexpr int KC = tc::KC<F16>;
    const int nrb_cap = (w.n + tc::TM - 1) / tc::TM;
    const int nkc_cap = (w.bmax + 1 + KC - 1) / KC;
    static int sms = 0;
    static bool attr = false;
    const size_t smem = (size_t)tc::STAGES * tc::STAGE_BYTES + 1024;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_trailing_kernel<F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long rows = (long long)w.n - kmin;
    const long long nrb = rows > 0 ? (rows + tc::TM - 1) / tc::TM : 1;
    cudaError_t e = launch_pdl(tc_prep_kernel<F16>, dim3(8 * sms), dim3(256), 0, s, w, ops, nrb_cap, nkc_cap);
    if (e != cudaSuccess) return e;
    count_launches(1);
    const long long tiles = supertile_count(nrb);
    const int grid = (int)(tiles < sms ? tiles : sms);
    e = launch_pdl(tc_trailing_kernel<F16>, dim3(grid > 0 ? grid : 1), dim3(TC_THREADS), smem, s, w, (const float *)ops,
                   nrb_cap, nkc_cap);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trailing_tc(const FactorWork<float> &w, float *ops, int kmin, bool f16, cudaStream_t s) {
    return f16 ? launch_trailing_tc_fmt<true>(w, ops, kmin, s) : launch_trailing_tc_fmt<false>(w, ops, kmin, s);
}

}  // namespace rcpk
