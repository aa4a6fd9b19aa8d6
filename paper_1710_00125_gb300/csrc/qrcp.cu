// qrcp.cu -- Algorithm 1 with q = b (Section 3.1, "Choosing q"): at the start of every block
// a b-step partial QR factorization with column pivoting (Businger-Golub: Householder
// reflections, the residual column norms recomputed at every step) of the sketch B(:, k0:n)
// chooses the block's pivot candidates, which are interchanged to positions k0, k0+1, ...; the
// block's pivot steps then take the column at position k instead of a sketch argmax, B is not
// updated inside the block, and after the block
//     B(:, k1:n) -= B(:, k0:k1) L11^{-T} L21^T
// (the block form of the sketch update, with L11 = L(k0:k1, k0:k1), L21 = L(k1:n, k0:k1) and
// B(:, k0:k1) the block-start sketch carried through the block's interchanges).
//
// qrcp_kernel is a cooperative kernel over the same CTA grid as the panel kernel: each CTA owns
// a chunk of the positions k0..n-1, keeps a working copy of their sketch columns in shared
// memory and tracks their current positions.  Per QRCP step every CTA publishes its best column
// (largest residual norm, smallest position on ties) with that column's residual part; after
// one grid barrier every CTA picks the winner, builds the same Householder vector from the
// winner's published residual and applies it to its own columns.  The resulting interchanges
// are written in the panel's format (lpos, moved list, an empty panel k0 = kend), so the
// interchange kernels apply them to A, the earlier L rows and perm; the sketch columns are
// moved here.
#include <type_traits>

#include "kernels.h"

namespace rcpk {

constexpr int QR_THREADS = 512;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr int QR_DMAX = 128;

template <typename T>
size_t qrcp_smem_bytes(int d, int chunk_cap) {
    return (size_t)chunk_cap * d * sizeof(T) + 2 * (size_t)chunk_cap * sizeof(int) + 64;
}

template <typename T>
__global__ void __launch_bounds__(QR_THREADS, 1) qrcp_kernel(FactorWork<T> w, int steps_max) {
    extern __shared__ __align__(16) unsigned char qr_smem[];
    __shared__ double s_wv[QR_WARPS];
    __shared__ int s_wp[QR_WARPS], s_wj[QR_WARPS];
    __shared__ T s_v[QR_DMAX];     // the Householder vector of the step (rows t..d-1)
    __shared__ double s_sc[4];     // ||x||, alpha, v^T v
    __shared__ int s_i[4];
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (ldcg(w.status) != 0) return;
    // this kernel's grid barriers advance the generation that indexes the panel's key rings
    // without clearing them: clear them here (no kernel reads them while this one runs)
    if (cta == 0)
        for (int e = tid; e < PANEL_KEY_WORDS; e += QR_THREADS) w.keys[e] = 0ull;
    const int n = w.n, d = w.d;
    const int k0 = ldcg(&w.st->next);
    if (k0 >= n) {
        if (cta == 0 && tid == 0) {
            w.st->n_moved = 0;
            w.st->k0 = n;
            w.st->kend = n;
        }
        return;
    }
    const int m = n - k0;
    const int chunk = (m + G - 1) / G;
    if (chunk > w.chunk_cap || d > QR_DMAX) {
        if (tid == 0) atomicOr(w.status, ST_INTERNAL);
        return;
    }
    const int j_lo = k0 + cta * chunk;
    const int cnt = max(0, min(n, j_lo + chunk) - j_lo);
    T *Wk = reinterpret_cast<T *>(qr_smem);                       // [cnt][d] working copy
    int *cur = reinterpret_cast<int *>(Wk + (size_t)w.chunk_cap * d);   // current positions
    int *chosen = cur + w.chunk_cap;
    for (int e = tid; e < cnt * d; e += QR_THREADS) {
        const int jl = e / d, r = e - jl * d;
        Wk[e] = w.B[(size_t)r + (size_t)(j_lo + jl) * d];
    }
    for (int jl = tid; jl < cnt; jl += QR_THREADS) {
        cur[jl] = j_lo + jl;
        chosen[jl] = 0;
    }
    if (tid == 0) {
        s_i[0] = (int)barrier_base(w.bar, (unsigned)G);
        if (cta == 0) w.st->n_moved = 0;
    }
    __syncthreads();
    const unsigned base = (unsigned)s_i[0];
    unsigned nbar = 0;
    double *rec = w.s1v;               // per CTA: residual norm^2, position (as double)
    T *pay = w.pay;                    // per CTA: the candidate's residual rows
    const int steps = min(min(steps_max, m), d);
    // The per-column work (residual norms, the reflection's dot products) runs in the factor's
    // type: FP32 factors take their QRCP decisions on FP32 values, as their panels do (and FP64
    // runs at 1/64 of the FP32 rate on this part); the few scalars of the reflection stay FP64.
    using R = T;
    for (int t = 0; t < steps; ++t) {
        // ---- the local candidate: largest residual norm over rows t..d-1 ----
        double bv = -1.0;
        int bp = INT_MAX, bj = -1;
        for (int jl = warp; jl < cnt; jl += QR_WARPS) {
            if (chosen[jl]) continue;
            R s2 = R(0);
            for (int r = t + lane; r < d; r += 32) {
                const R x = (R)Wk[(size_t)jl * d + r];
                s2 += x * x;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
            const double s2d = (double)s2;
            if (s2d > bv || (s2d == bv && cur[jl] < bp)) { bv = s2d; bp = cur[jl]; bj = jl; }
        }
        if (lane == 0) { s_wv[warp] = bv; s_wp[warp] = bp; s_wj[warp] = bj; }
        __syncthreads();
        if (tid == 0) {
            for (int q = 1; q < QR_WARPS; ++q)
                if (s_wv[q] > bv || (s_wv[q] == bv && s_wp[q] < bp)) { bv = s_wv[q]; bp = s_wp[q]; bj = s_wj[q]; }
            stcg(reinterpret_cast<double2 *>(rec + 4 * (size_t)cta), make_double2(bv, (double)bp));
            s_i[1] = bj;
        }
        __syncthreads();
        if (s_i[1] >= 0)
            for (int r = t + tid; r < d; r += QR_THREADS) stcg(pay + (size_t)cta * d + r, Wk[(size_t)s_i[1] * d + r]);
        if (!grid_barrier(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
        // ---- the winner (every CTA reduces the same records in the same order) ----
        if (warp == 0) {
            double v = -1.0;
            int p = INT_MAX, g = -1;
            for (int q = lane; q < G; q += 32) {
                const double2 x = __ldcg(reinterpret_cast<const double2 *>(rec + 4 * (size_t)q));
                const int xp = (int)x.y;
                if (x.x > v || (x.x == v && xp < p)) { v = x.x; p = xp; g = q; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, v, off);
                const int p2 = __shfl_xor_sync(0xffffffffu, p, off), g2 = __shfl_xor_sync(0xffffffffu, g, off);
                if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; g = g2; }
            }
            if (lane == 0) { s_i[2] = p; s_i[3] = g; }
        }
        __syncthreads();
        const int wpos = s_i[2], wcta = s_i[3];
        if (wcta < 0 || wpos < k0 + t || wpos >= n) {
            // no finite residual norm left (NaN or Inf in the sketch)
            if (tid == 0) atomicOr(w.status, ST_NONFINITE);
            return;
        }
        for (int r = t + tid; r < d; r += QR_THREADS) s_v[r] = ldcg(pay + (size_t)wcta * d + r);
        // ---- interchange k0 + t <-> wpos in the owned bookkeeping ----
        for (int jl = tid; jl < cnt; jl += QR_THREADS) {
            const int o = cur[jl];
            if (o == wpos) { cur[jl] = k0 + t; chosen[jl] = 1; }
            else if (o == k0 + t) cur[jl] = wpos;
        }
        __syncthreads();
        // ---- the Householder reflection zeroing x(t+1:d) (same arithmetic in every CTA) ----
        if (warp == 0) {
            double s2 = 0.0;
            for (int r = t + lane; r < d; r += 32) s2 += (double)s_v[r] * (double)s_v[r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
            if (lane == 0) {
                const double nrm = sqrt(s2), x0 = (double)s_v[t];
                const double alpha = x0 >= 0.0 ? -nrm : nrm;
                s_sc[0] = nrm;
                s_sc[1] = alpha;
                s_v[t] = (T)(x0 - alpha);
            }
            __syncwarp();
            double vv = 0.0;
            for (int r = t + lane; r < d; r += 32) vv += (double)s_v[r] * (double)s_v[r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, off);
            if (lane == 0) {
                s_sc[2] = vv;
                s_sc[3] = vv > 0.0 ? 2.0 / vv : 0.0;
            }
        }
        __syncthreads();
        if (s_sc[0] != 0.0 && s_sc[2] > 0.0) {
            const double vv = s_sc[2];
            for (int jl = warp; jl < cnt; jl += QR_WARPS) {
                if (chosen[jl]) continue;
                T *col = Wk + (size_t)jl * d;
                R dot = R(0);
                for (int r = t + lane; r < d; r += 32) dot += (R)s_v[r] * (R)col[r];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
                T f;
                if constexpr (sizeof(T) == sizeof(double)) f = (T)(2.0 * dot / vv);
                else f = dot * (T)s_sc[3];   // 2 / v^T v, formed once per step
                for (int r = t + lane; r < d; r += 32) col[r] -= f * s_v[r];
            }
        }
        __syncthreads();
    }
    // ---- publish the interchanges in the panel's format; move the sketch columns ----
    for (int jl = tid; jl < cnt; jl += QR_THREADS) {
        const int j = j_lo + jl;
        w.lpos[j] = cur[jl];
        chosen[jl] = -1;
        if (cur[jl] != j) {
            const int idx = atomicAdd(&w.st->n_moved, 1);
            if (idx < w.maxmoved) {
                w.moved[idx] = j;
                chosen[jl] = idx;
            } else {
                atomicOr(w.status, ST_INTERNAL);
            }
        }
    }
    __syncthreads();
    // original columns of the moved indices to scratch (B itself is still untouched), then to
    // their new positions after the barrier
    for (int jl = warp; jl < cnt; jl += QR_WARPS) {
        const int idx = chosen[jl];
        if (idx < 0) continue;
        for (int r = lane; r < d; r += 32) w.tmpA[(size_t)idx * d + r] = w.B[(size_t)r + (size_t)(j_lo + jl) * d];
    }
    if (!grid_barrier(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
    for (int jl = warp; jl < cnt; jl += QR_WARPS) {
        const int idx = chosen[jl];
        if (idx < 0) continue;
        for (int r = lane; r < d; r += 32) w.B[(size_t)r + (size_t)cur[jl] * d] = ldcg(w.tmpA + (size_t)idx * d + r);
    }
    if (cta == 0 && tid == 0) {
        w.st->k0 = k0;
        w.st->kend = k0;
    }
}

// The FP32 block QRCP, arranged around one exchange per step like the FP32 panel: the step's
// reflection, the downdated residual norms (recomputed from the updated rows t+1..d-1) and the
// CTA's next candidate come out of one pass over the owned columns, four threads per column (a
// quad: rows t + sub, t + sub + 4, ...; two shuffles per reduction); the candidates meet in one
// packed 64-bit key per CTA (norm bits, inverted position, CTA) folded by red.max into the
// panel's key ring, and after the grid barrier a single key load names the winner, whose
// residual rows the winning CTA published beside it.  The reflection's scalars are formed in
// FP32, the factor's type (an FP32 factor takes its pivot decisions on FP32 values).
__device__ __forceinline__ unsigned long long qr_block_max(unsigned long long v, unsigned long long *slots) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_max_u64(v);
    if (lane == 0) slots[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = warp_max_u64(lane < QR_WARPS ? slots[lane] : 0ull);
        if (lane == 0) slots[QR_WARPS] = x;
    }
    __syncthreads();
    return slots[QR_WARPS];
}

__global__ void __launch_bounds__(QR_THREADS, 1) qrcp_keys_kernel(FactorWork<float> w, int steps_max) {
    extern __shared__ __align__(16) unsigned char qr_smem[];
    __shared__ unsigned long long s_slots[QR_WARPS + 1];
    __shared__ float s_v[QR_DMAX];   // the Householder vector of the step (rows t..d-1)
    __shared__ double s_sc[4];       // ||x||, alpha, v^T v, 2 / v^T v
    __shared__ int s_i[4];
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (ldcg(w.status) != 0) return;
    const int n = w.n, d = w.d;
    const int k0 = ldcg(&w.st->next);
    if (k0 >= n) {
        if (cta == 0 && tid == 0) {
            w.st->n_moved = 0;
            w.st->k0 = n;
            w.st->kend = n;
        }
        return;
    }
    const int m = n - k0;
    const int chunk = (m + G - 1) / G;
    if (chunk > w.chunk_cap || d > QR_DMAX || G > 0xFFFF) {
        if (tid == 0) atomicOr(w.status, ST_INTERNAL);
        return;
    }
    const int j_lo = k0 + cta * chunk;
    const int cnt = max(0, min(n, j_lo + chunk) - j_lo);
    float *Wk = reinterpret_cast<float *>(qr_smem);                     // [cnt][d] working copy
    int *cur = reinterpret_cast<int *>(Wk + (size_t)w.chunk_cap * d);   // current positions
    int *chosen = cur + w.chunk_cap;
    for (int e = tid; e < cnt * d; e += QR_THREADS) {
        const int jl = e / d, r = e - jl * d;
        Wk[e] = w.B[(size_t)r + (size_t)(j_lo + jl) * d];
    }
    for (int jl = tid; jl < cnt; jl += QR_THREADS) {
        cur[jl] = j_lo + jl;
        chosen[jl] = 0;
    }
    if (tid == 0) {
        s_i[0] = (int)barrier_base(w.bar, (unsigned)G);
        if (cta == 0) w.st->n_moved = 0;
    }
    __syncthreads();
    const unsigned base = (unsigned)s_i[0];
    const unsigned gbase = base / (unsigned)G;
    unsigned nbar = 0;
    float *pay = w.pay;   // per CTA: the candidate's residual rows
    unsigned long long *keys = w.keys;
    const int steps = min(min(steps_max, m), d);
    // the CTA's candidate for step 0: largest ||B(:, j)||^2 (local key: norm bits, position, index)
    constexpr int QUADS = QR_THREADS / 4;
    const int quad = tid >> 2, sub = tid & 3;
    unsigned long long key = 0ull;
    for (int jl0 = 0; jl0 < cnt; jl0 += QUADS) {
        const int jl = jl0 + quad;
        float s2 = 0.f;
        if (jl < cnt)
            for (int r = sub; r < d; r += 4) {
                const float x = Wk[(size_t)jl * d + r];
                s2 = fmaf(x, x, s2);
            }
        s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
        s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
        if (jl < cnt && sub == 0) key = max(key, make_key(s2, cur[jl], jl));
    }
    for (int t = 0; t < steps; ++t) {
        const unsigned long long kc = qr_block_max(key, s_slots);
        const unsigned g = gbase + nbar + 1;
        if (kc != 0ull) {
            const int jc = (int)(kc & 0xFFFFull);
            for (int r = t + tid; r < d; r += QR_THREADS) stcg(pay + (size_t)cta * d + r, Wk[(size_t)jc * d + r]);
            if (tid == 0) red_max_u64(key_slot(keys, g), (kc & ~0xFFFFull) | (unsigned long long)cta);
        }
        if (!grid_barrier(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
        if (tid == 0) {
            const unsigned long long kw = ld_key(key_slot(keys, g));
            if (cta == 0) *key_slot(keys, g + KEY_RING / 2) = 0ull;
            const float v = __uint_as_float((unsigned)(kw >> 32));
            s_i[2] = kw != 0ull && isfinite(v) ? 0xFFFF - (int)((kw >> 16) & 0xFFFFull) : -1;
            s_i[3] = (int)(kw & 0xFFFFull);
        }
        __syncthreads();
        const int wpos = s_i[2], wcta = s_i[3];
        if (wpos < k0 + t || wpos >= n || wcta >= G) {
            // no finite residual norm left (NaN or Inf in the sketch)
            if (tid == 0) atomicOr(w.status, ST_NONFINITE);
            return;
        }
        for (int r = t + tid; r < d; r += QR_THREADS) s_v[r] = ldcg(pay + (size_t)wcta * d + r);
        // ---- interchange k0 + t <-> wpos in the owned bookkeeping ----
        for (int jl = tid; jl < cnt; jl += QR_THREADS) {
            const int o = cur[jl];
            if (o == wpos) { cur[jl] = k0 + t; chosen[jl] = 1; }
            else if (o == k0 + t) cur[jl] = wpos;
        }
        __syncthreads();
        // ---- the Householder reflection zeroing x(t+1:d) (same arithmetic in every CTA) ----
        if (warp == 0) {
            float s2 = 0.f;
            for (int r = t + lane; r < d; r += 32) s2 = fmaf(s_v[r], s_v[r], s2);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
            const float nrm = sqrtf(s2), x0 = s_v[t];
            const float alpha = x0 >= 0.f ? -nrm : nrm;
            __syncwarp();
            if (lane == 0) s_v[t] = x0 - alpha;
            __syncwarp();
            float vv = 0.f;
            for (int r = t + lane; r < d; r += 32) vv = fmaf(s_v[r], s_v[r], vv);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, off);
            if (lane == 0) {
                s_sc[0] = nrm;
                s_sc[2] = vv;
                s_sc[3] = vv > 0.f ? 2.f / vv : 0.f;
            }
        }
        __syncthreads();
        // ---- the reflection on every owned column left, its residual norm over rows t+1..d-1
        // and the CTA's candidate for the next step, in one pass (a quad per column) ----
        const bool reflect = s_sc[0] != 0.0 && s_sc[2] > 0.0;
        const float f2 = (float)s_sc[3];
        key = 0ull;
        for (int jl0 = 0; jl0 < cnt; jl0 += QUADS) {
            const int jl = jl0 + quad;
            const bool live = jl < cnt && !chosen[jl];
            float *col = Wk + (size_t)(live ? jl : 0) * d;
            float dot = 0.f;
            if (live && reflect)
                for (int r = t + sub; r < d; r += 4) dot = fmaf(s_v[r], col[r], dot);
            dot += __shfl_xor_sync(0xffffffffu, dot, 1);
            dot += __shfl_xor_sync(0xffffffffu, dot, 2);
            float s2 = 0.f;
            if (live) {
                const float f = dot * f2;
                for (int r = t + sub; r < d; r += 4) {
                    float x = col[r];
                    if (reflect) {
                        x = fmaf(-f, s_v[r], x);
                        col[r] = x;
                    }
                    if (r > t) s2 = fmaf(x, x, s2);   // rows t+1.. are the next step's residual
                }
            }
            s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
            s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
            if (live && sub == 0) key = max(key, make_key(s2, cur[jl], jl));
        }
        __syncthreads();
    }
    // ---- publish the interchanges in the panel's format; move the sketch columns ----
    for (int jl = tid; jl < cnt; jl += QR_THREADS) {
        const int j = j_lo + jl;
        w.lpos[j] = cur[jl];
        chosen[jl] = -1;
        if (cur[jl] != j) {
            const int idx = atomicAdd(&w.st->n_moved, 1);
            if (idx < w.maxmoved) {
                w.moved[idx] = j;
                chosen[jl] = idx;
            } else {
                atomicOr(w.status, ST_INTERNAL);
            }
        }
    }
    __syncthreads();
    for (int jl = warp; jl < cnt; jl += QR_WARPS) {
        const int idx = chosen[jl];
        if (idx < 0) continue;
        for (int r = lane; r < d; r += 32) w.tmpA[(size_t)idx * d + r] = w.B[(size_t)r + (size_t)(j_lo + jl) * d];
    }
    {
        const unsigned g = gbase + nbar + 1;
        if (!grid_barrier(w.bar, base + (++nbar) * (unsigned)G, w.status)) return;
        if (cta == 0 && tid == 0) *key_slot(keys, g + KEY_RING / 2) = 0ull;   // the ring stays in step
    }
    for (int jl = warp; jl < cnt; jl += QR_WARPS) {
        const int idx = chosen[jl];
        if (idx < 0) continue;
        for (int r = lane; r < d; r += 32) w.B[(size_t)r + (size_t)cur[jl] * d] = ldcg(w.tmpA + (size_t)idx * d + r);
    }
    if (cta == 0 && tid == 0) {
        w.st->k0 = k0;
        w.st->kend = k0;
    }
}

// Y = B(:, k0:k1) L11^{-T} (Y L11^T = B(:, blk), column by column), one CTA; Y^T is kept in
// shared memory as [c][r] and written to ytmp (d x nb, ld d).
template <typename T>
__global__ void __launch_bounds__(1024) bsk_y_kernel(FactorWork<T> w, T *ytmp) {
    extern __shared__ __align__(16) unsigned char by_smem[];
    if (ldcg(w.status) != 0) return;
    const int n = w.n, d = w.d, k0 = w.st->k0, k1 = w.st->kend, nb = k1 - k0;
    if (nb <= 0 || k1 >= n) return;
    T *Yt = reinterpret_cast<T *>(by_smem);   // [nb][d]
    for (int e = threadIdx.x; e < nb * d; e += blockDim.x) {
        const int c = e / d, r = e - c * d;
        Yt[e] = w.B[(size_t)r + (size_t)(k0 + c) * d];
    }
    __syncthreads();
    // forward substitution with the unit lower L11: row c of Y^T is final once the rows
    // before it have been subtracted; then it updates the rows below
    for (int c = 0; c < nb - 1; ++c) {
        const int rows = nb - c - 1;
        for (int e = threadIdx.x; e < rows * d; e += blockDim.x) {
            const int c2 = c + 1 + e / d, r = e % d;
            const T l = w.Lc[(size_t)(k0 + c2) + (size_t)c * n];
            Yt[(size_t)c2 * d + r] -= l * Yt[(size_t)c * d + r];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * d; e += blockDim.x) {
        const int c = e / d, r = e - c * d;
        ytmp[(size_t)r + (size_t)c * d] = Yt[e];
    }
}

// B(r, j) -= sum_c Y(r, c) L(j, k0 + c), j >= k1: CTA over 128 columns j and 16 rows r.
template <typename T>
__global__ void __launch_bounds__(128) bsk_update_kernel(FactorWork<T> w, const T *ytmp) {
    extern __shared__ __align__(16) unsigned char bu_smem[];
    if (ldcg(w.status) != 0) return;
    const int n = w.n, d = w.d, k0 = w.st->k0, k1 = w.st->kend, nb = k1 - k0;
    if (nb <= 0 || k1 >= n) return;
    T *Ys = reinterpret_cast<T *>(bu_smem);   // [16][nb]
    const int r0 = blockIdx.y * 16, rr = min(16, d - r0);
    for (int e = threadIdx.x; e < 16 * nb; e += blockDim.x) {
        const int q = e / nb, c = e - q * nb;
        Ys[e] = q < rr ? ytmp[(size_t)(r0 + q) + (size_t)c * d] : T(0);
    }
    __syncthreads();
    const int j = k1 + blockIdx.x * 128 + threadIdx.x;
    if (j >= n) return;
    T acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = T(0);
    for (int c = 0; c < nb; ++c) {
        const T l = w.Lc[(size_t)j + (size_t)c * n];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] += Ys[q * nb + c] * l;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (q < rr) w.B[(size_t)(r0 + q) + (size_t)j * d] -= acc[q];
}

template <typename T>
cudaError_t launch_qrcp(const FactorWork<T> &w, int steps, cudaStream_t s) {
    const size_t smem = qrcp_smem_bytes<T>(w.d, w.chunk_cap);
    // FP32: the key-exchange kernel (it keeps the panel's key ring in step, so the ring must
    // have been zeroed at the start of the factorization, as factor_impl does)
    const void *fn = std::is_same<T, float>::value ? (const void *)qrcp_keys_kernel : (const void *)qrcp_kernel<T>;
    static int attr_set = 0;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = 1;
    }
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    FactorWork<T> arg = w;
    int st = steps;
    void *args[] = {&arg, &st};
    count_launches(1);
    return cudaLaunchCooperativeKernel(fn, dim3(w.grid), dim3(QR_THREADS), args, smem, s);
}

template <typename T>
cudaError_t launch_bsk_y(const FactorWork<T> &w, T *ytmp, cudaStream_t s) {
    const size_t ysm = (size_t)w.bw * w.d * sizeof(T);
    static int attr_set = 0;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(bsk_y_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = 1;
    }
    if (ysm > 200 * 1024) return cudaErrorInvalidValue;
    bsk_y_kernel<T><<<1, 1024, ysm, s>>>(w, ytmp);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_block_sketch_update(const FactorWork<T> &w, T *ytmp, cudaStream_t s) {
    const size_t ysm = (size_t)w.bw * w.d * sizeof(T), usm = (size_t)16 * w.bw * sizeof(T);
    static int attr_set = 0;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(bsk_y_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(bsk_update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = 1;
    }
    if (ysm > 200 * 1024 || usm > 200 * 1024) return cudaErrorInvalidValue;
    bsk_y_kernel<T><<<1, 1024, ysm, s>>>(w, ytmp);
    count_launches(1);
    dim3 g((w.n + 127) / 128, (w.d + 15) / 16);
    bsk_update_kernel<T><<<g, 128, usm, s>>>(w, ytmp);
    count_launches(1);
    return cudaGetLastError();
}

size_t qrcp_smem_limit() { return 200 * 1024; }

template size_t qrcp_smem_bytes<double>(int, int);
template size_t qrcp_smem_bytes<float>(int, int);
template cudaError_t launch_qrcp<double>(const FactorWork<double> &, int, cudaStream_t);
template cudaError_t launch_qrcp<float>(const FactorWork<float> &, int, cudaStream_t);
template cudaError_t launch_bsk_y<double>(const FactorWork<double> &, double *, cudaStream_t);
template cudaError_t launch_bsk_y<float>(const FactorWork<float> &, float *, cudaStream_t);
template cudaError_t launch_block_sketch_update<double>(const FactorWork<double> &, double *, cudaStream_t);
template cudaError_t launch_block_sketch_update<float>(const FactorWork<float> &, float *, cudaStream_t);

}  // namespace rcpk
