// rcp_api.cu -- the C ABI declared in include/rcp.h: handle, workspace and the host-side
// orchestration of the kernels on one CUDA stream.  In the factorization, the solves and the
// classic refinement, loop control that depends on data (panel widths, refinement convergence)
// stays on the device, so the launch sequence of a call depends only on its arguments.  The
// host-driven calls read device scalars between launches: GMRES-based refinement (the Krylov
// least-squares problem), the factorization with the Algorithm 2 safeguard (one state read per
// panel) and the 1-norm estimator of rcp_l_norms.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <type_traits>
#include <vector>

#include "../../include/rcp.h"
#include "kernels.h"

using namespace rcpk;

namespace rcpk {
static std::atomic<long long> g_launches{0};
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace rcpk

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

// PH_H2D: rcp_sysv's host-to-device copies with host buffers, bracketed on the stream that
// issues them (the copy stream for FP32 factors, where they overlap the sketch)
enum Phase { PH_SKETCH = 0, PH_PANEL, PH_INTERCHANGE, PH_TRAILING, PH_SOLVE, PH_RESIDUAL, PH_H2D, PH_COUNT };

struct EventPair {
    int phase;
    cudaEvent_t a, b;
};

struct rcp_handle {
    int device = 0;
    int profiling = 0;
    int spec_mode = -1;                            // FP32 panel speculation (rcp_set_speculation)
    std::vector<EventPair> events;      // recorded pairs of the calls since the last read
    std::vector<cudaEvent_t> pool;      // free events
    int launches[PH_COUNT] = {0};
    Buf status, state, bar, scal;                 // small persistent buffers
    Buf om, B, Wbuf, Lc, Lg, lpos, moved, s1v, s2v, s3v, s1i, s2i, pay, tmpA, tmpL, tmpP;
    Buf Y, flags, R, Dc, part;
    Buf A64, F, Bh, Xh, Dd, Ds, perm;              // rcp_sysv buffers
    Buf trace;                                     // per-step panel timestamps (profiling level 2)
    Buf psnap, pinv, pbounds;                      // deferred L-row interchanges
    Buf keys;                                      // packed argmax keys of the FP32 panel
    Buf skp;                                       // partial sums of the FP32 sketch
    Buf omt;                                       // Omega split into TF32 tiles (tensor-core sketch)
    Buf tcops;                                     // tensor-core operand tiles
    int trace_n = 0;
    Buf bord, bom, bticket, bscr;                  // batched path: order, Omega, ticket, per-CTA scratch
    const int *bord_n = nullptr;                   // (n, batch, nmax) the order was made for
    int bord_batch = -1, bord_nmax = -1;
    uint64_t bom_seed = 0;                         // (seed, d, nmax, fp64) of the drawn Omega
    int bom_d = -1, bom_nmax = -1, bom_f64 = -1;
    struct Tuned { int nmax, dkey, f64, b, d, nt, split; };   // dkey: the caller's d (0: d = b + 8 tuned with b)
    std::vector<Tuned> tuned;                      // batched shapes chosen by rcp_tune_batched
    int bt_nt = 0, bt_split = 0;                   // rcp_set_batched_schedule (0, 0: tuned or default)
    cudaStream_t copy_stream = nullptr;            // rcp_sysv with host buffers: block copies of A
    std::vector<cudaEvent_t> copy_events;          //   one per block, and one for the start
    Buf gmV, gmZ, gmP, gmH;                        // GMRES refinement: basis, zero vector, partial sums, scalars
    Buf iperm;                                     // identity permutation (one-triangle solves)
};

namespace {

// grow(), and zero the buffer (on stream s, or synchronously when s is null) when it was
// reallocated
rcp_status grow_zeroed(Buf &b, size_t bytes, cudaStream_t s, bool sync);

rcp_status grow(Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return RCP_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RCP_ENOMEM;
    }
    b.bytes = bytes;
    return RCP_OK;
}

rcp_status grow_zeroed(Buf &b, size_t bytes, cudaStream_t s, bool sync) {
    void *old = b.p;
    const size_t had = b.bytes;
    const rcp_status g = grow(b, bytes);
    if (g != RCP_OK) return g;
    if (b.p != old || b.bytes != had) {
        if (sync) {
            if (cudaMemset(b.p, 0, b.bytes) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return RCP_ECUDA;
        } else if (cudaMemsetAsync(b.p, 0, b.bytes, s) != cudaSuccess) {
            return RCP_ECUDA;
        }
    }
    return RCP_OK;
}

#define RCP_TRY(x)                          \
    do {                                    \
        rcp_status _s = (x);                \
        if (_s != RCP_OK) return _s;        \
    } while (0)
#define CU_TRY(x)                           \
    do {                                    \
        if ((x) != cudaSuccess) {           \
            cudaGetLastError();             \
            return RCP_ECUDA;               \
        }                                   \
    } while (0)

// Scalars of the refinement loop, laid out in h->scal.
struct RefineScalars {
    int conv;               // 0 running, 1 converged, 2 stopped: a correction did not halve berr
    int iters;
    double prev;            // berr of the previous iterate (0 before the first)
    double berr;
    double anorm;
    unsigned long long mx[2 * 1024];   // per right-hand side: max |r|, max |x|
};
constexpr int kMaxRhs = 1024;

rcp_status ensure_small(rcp_handle *h) {
    bool fresh = h->status.p == nullptr;
    RCP_TRY(grow(h->status, 64));
    RCP_TRY(grow(h->state, sizeof(FactorState)));
    RCP_TRY(grow(h->bar, 64));
    RCP_TRY(grow(h->scal, sizeof(RefineScalars)));
    if (fresh) {
        CU_TRY(cudaMemset(h->status.p, 0, 64));
        CU_TRY(cudaMemset(h->bar.p, 0, 64));
    }
    return RCP_OK;
}

bool tc_prec(rcp_prec p) { return p == RCP_TF32X3 || p == RCP_F16X3; }

struct Resolved {
    int b, d, grid, chunk_cap, bw, maxmoved, spec, qb;
    int guard_r;           // Algorithm 2 (0 = off)
    double guard_eps;
    double alpha;
    rcp_prec prec;
    uint64_t seed;
    const void *omega;
};

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

rcp_status resolve(int n, const rcp_opts *o, Resolved &r, int spec_mode = -1) {
    r.prec = o ? o->prec : RCP_FP64;
    if (r.prec < RCP_FP64 || r.prec > RCP_F16X3) return RCP_EINVAL;
    r.b = (o && o->b > 0) ? o->b : 64;
    r.d = (o && o->d > 0) ? o->d : std::min(r.b + 16, 128);
    if (o && (o->q_mode < 0 || o->q_mode > 2)) return RCP_EUNSUPPORTED;
    r.qb = (o && o->q_mode == 2) ? 1 : 0;
    if (r.b < 1 || r.b > 512 || r.d < 1 || r.d > 128) return RCP_EUNSUPPORTED;
    r.alpha = (o && o->alpha > 0.0) ? o->alpha : std::sqrt(2.0) / 2.0;
    if (!(r.alpha < 1.0)) return RCP_EINVAL;
    r.seed = o ? o->seed : 0;
    r.omega = o ? o->omega : nullptr;
    r.guard_r = o ? o->guard_r : 0;
    if (r.guard_r < 0 || r.guard_r > 64) return RCP_EINVAL;
    r.guard_eps = (o && o->guard_eps > 0.0) ? o->guard_eps
                                            : (r.prec == RCP_FP64 ? 0x1.0p-52 : 0x1.0p-23);   // machine epsilon
    if (!(r.guard_eps < 1.0)) return RCP_EINVAL;
    if (r.guard_r > 0 && r.qb) return RCP_EUNSUPPORTED;   // the safeguard is defined for q = 1
    r.bw = r.b + 1;
    // each pivot column costs at most two transpositions, and each moves two indices
    r.maxmoved = 4 * (r.b + 2);
    const bool f64 = r.prec == RCP_FP64;
    if (!f64 && n > 65535) return RCP_EUNSUPPORTED;   // positions and indices are packed in 16 bits
    int maxg = 0;
    int sms = sm_count();
    int g = (o && o->grid > 0) ? o->grid : std::min(sms, std::max(1, (n + 31) / 32));
    if (n > 0) g = std::min(g, n);
    g = std::max(1, g);
    r.chunk_cap = (n + g - 1) / g;
    if (r.chunk_cap > 1024) return RCP_EUNSUPPORTED;
    // the FP32 panel speculates on SBKP case (1): with a shadow copy of its sketch columns when that
    // fits in shared memory, else with the sketch update deferred to the next step's pass
    r.spec = 0;
    if (r.qb) {
        // q = b: the block QRCP keeps its chunk of the sketch in shared memory, and the block
        // sketch update keeps Y^T (bw x d) there; no speculation (no per-step sketch argmax)
        const size_t el = f64 ? sizeof(double) : sizeof(float);
        if ((f64 ? qrcp_smem_bytes<double>(r.d, r.chunk_cap) : qrcp_smem_bytes<float>(r.d, r.chunk_cap)) >
                qrcp_smem_limit() ||
            (size_t)r.bw * r.d * el > qrcp_smem_limit())
            return RCP_EUNSUPPORTED;
        maxg = f64 ? panel_max_grid<double>(r.d, r.bw, r.chunk_cap, 0) : panel_max_grid<float>(r.d, r.bw, r.chunk_cap, 0);
    } else if (f64) {
        maxg = panel_max_grid<double>(r.d, r.bw, r.chunk_cap, 0);
    } else {
        // speculation with the shadow sketch (1), else with the deferred sketch update (2), else
        // none; spec_mode forces one of them (-1: this order)
        if (spec_mode == -1 || spec_mode == 1) {
            const int m1 = panel_max_grid<float>(r.d, r.bw, r.chunk_cap, 1);
            if (m1 >= g) { r.spec = 1; maxg = m1; }
        }
        if (r.spec == 0 && (spec_mode == -1 || spec_mode == 2)) {
            const int m2 = panel_max_grid<float>(r.d, r.bw, r.chunk_cap, 2);
            if (m2 >= g) { r.spec = 2; maxg = m2; }
        }
        if (r.spec == 0) {
            if (spec_mode == 1 || spec_mode == 2) return RCP_EUNSUPPORTED;
            maxg = panel_max_grid<float>(r.d, r.bw, r.chunk_cap, 0);
        }
    }
    if (maxg <= 0 || g > maxg) return RCP_EUNSUPPORTED;
    r.grid = g;
    return RCP_OK;
}

template <typename T>
rcp_status ensure_factor_ws(rcp_handle *h, int n, const Resolved &r) {
    RCP_TRY(ensure_small(h));
    const size_t N = n > 0 ? n : 1;
    RCP_TRY(grow(h->om, N * r.d * sizeof(T)));
    RCP_TRY(grow(h->B, N * r.d * sizeof(T)));
    RCP_TRY(grow(h->Wbuf, N * r.bw * sizeof(T)));
    RCP_TRY(grow(h->Lc, N * r.bw * sizeof(T)));
    RCP_TRY(grow(h->Lg, N * r.bw * sizeof(T)));
    RCP_TRY(grow(h->lpos, N * sizeof(int)));
    RCP_TRY(grow(h->moved, 2 * N * sizeof(int)));
    RCP_TRY(grow(h->s1v, 4 * (size_t)r.grid * sizeof(double)));
    RCP_TRY(grow(h->s2v, 4 * (size_t)r.grid * sizeof(double)));
    RCP_TRY(grow(h->keys, PANEL_KEY_WORDS * sizeof(unsigned long long)));
    if (sizeof(T) == sizeof(float))
        RCP_TRY(grow(h->skp, std::max(sketch_scratch_floats(n, r.d), sketch_tc_scratch_floats(n, r.d)) * sizeof(float)));
    if (tc_prec(r.prec))   // Omega's tiles for the sketch, later Y's for the q = b block update
        RCP_TRY(grow(h->omt, std::max(sketch_tc_omega_floats(n, r.d), block_update_tc_floats(r.bw, r.d)) * sizeof(float)));
    if (r.prec == RCP_TF32X3 || r.prec == RCP_F16X3) RCP_TRY(grow(h->tcops, tc_ops_floats(n, r.b) * sizeof(float)));
    RCP_TRY(grow(h->s1i, 2 * (size_t)r.grid * sizeof(int)));
    RCP_TRY(grow(h->s2i, 2 * (size_t)r.grid * sizeof(int)));
    RCP_TRY(grow(h->pay, 4 * (size_t)r.grid * r.d * sizeof(T)));
    RCP_TRY(grow(h->s3v, 8 * (size_t)r.grid * sizeof(double)));
    // interchange scratch; with q = b it also holds the moved sketch columns and Y (d x bw)
    const size_t NT = std::max(N, (size_t)r.d);
    RCP_TRY(grow(h->tmpA, (size_t)r.maxmoved * NT * sizeof(T)));
    RCP_TRY(grow(h->tmpL, (size_t)r.maxmoved * NT * sizeof(T)));
    RCP_TRY(grow(h->tmpP, (size_t)r.maxmoved * sizeof(int)));
    // each safeguard event ends a panel early: at most guard_r panels more
    const size_t npan = (N + r.b - 1) / r.b + (size_t)r.guard_r;
    RCP_TRY(grow(h->psnap, npan * N * sizeof(int)));
    RCP_TRY(grow(h->pinv, npan * N * sizeof(int)));
    RCP_TRY(grow(h->pbounds, 2 * npan * sizeof(int)));
    return RCP_OK;
}

template <typename T>
FactorWork<T> make_work(rcp_handle *h, int n, T *A, int lda, double *Dd, double *Ds, int *perm, const Resolved &r) {
    FactorWork<T> w;
    w.n = n; w.lda = lda; w.A = A;
    w.d = r.d; w.B = (T *)h->B.p;
    w.bmax = r.b; w.bw = r.bw; w.alpha = r.alpha;
    w.Wbuf = (T *)h->Wbuf.p; w.Lc = (T *)h->Lc.p; w.Lg = (T *)h->Lg.p;
    w.Dd = Dd; w.Ds = Ds; w.perm = perm;
    w.lpos = (int *)h->lpos.p; w.moved = (int *)h->moved.p;
    w.st = (FactorState *)h->state.p;
    w.s1v = (double *)h->s1v.p; w.s2v = (double *)h->s2v.p;
    w.s1i = (int *)h->s1i.p; w.s2i = (int *)h->s2i.p;
    w.pay = (T *)h->pay.p;
    w.bar = (unsigned *)h->bar.p;
    w.status = (int *)h->status.p;
    w.grid = r.grid; w.chunk_cap = r.chunk_cap;
    w.tmpA = (T *)h->tmpA.p; w.tmpL = (T *)h->tmpL.p; w.tmpP = (int *)h->tmpP.p;
    w.maxmoved = r.maxmoved;
    w.keys = (unsigned long long *)h->keys.p;
    w.spec = r.spec;
    w.qb = r.qb;
    w.guard_r = r.guard_r;
    w.guard_eps = r.guard_eps;
    w.psnap = (int *)h->psnap.p;
    w.pinv = (int *)h->pinv.p;
    w.pbounds = (int *)h->pbounds.p;
    w.s3v = (double *)h->s3v.p;
    w.tcops = (r.prec == RCP_TF32X3 || r.prec == RCP_F16X3) ? (float *)h->tcops.p : nullptr;
    w.trace = nullptr;
    if (h->profiling >= 2 && grow(h->trace, (size_t)n * PANEL_TRACE_SLOTS * sizeof(unsigned long long)) == RCP_OK) {
        w.trace = (unsigned long long *)h->trace.p;
        cudaMemset(h->trace.p, 0, (size_t)n * PANEL_TRACE_SLOTS * sizeof(unsigned long long));
        h->trace_n = n;
    }
    return w;
}

rcp_status status_from_bits(int bits) {
    if (bits & ST_TIMEOUT) return RCP_ETIMEOUT;
    if (bits & ST_NONFINITE) return RCP_ENONFINITE;
    if (bits & ST_INTERNAL) return RCP_ECUDA;
    return RCP_OK;
}

cudaEvent_t take_event(rcp_handle *h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets a stretch of launches of one phase with two events when profiling is on.
struct PhaseScope {
    rcp_handle *h;
    cudaStream_t s;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseScope(rcp_handle *h_, cudaStream_t s_, int ph) : h(h_), s(s_), phase(ph) {
        if (h->profiling) {
            a = take_event(h);
            cudaEventRecord(a, s);
        }
    }
    ~PhaseScope() {
        if (h->profiling && a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, s);
            h->events.push_back({phase, a, b});
            h->launches[phase] += 1;
        }
    }
};

// column block of the host-to-device copy of A in rcp_sysv (host_buffers)
constexpr int kHostCopyCols = 256;

double bits_to_double(unsigned long long b) {
    double v;
    std::memcpy(&v, &b, sizeof v);
    return v;
}

// B = Omega A (d x n) of the order-n matrix A in the factor's arithmetic: FP64 or FP32 on the
// CUDA cores, the tensor-core precisions by the split-TF32 tcgen05 sketch
template <typename T>
cudaError_t sketch_for(rcp_handle *h, const Resolved &r, int n, const T *A, int lda, const T *om, T *B, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (tc_prec(r.prec)) {
            cudaError_t e = launch_omega_split(n, r.d, om, (float *)h->omt.p, s);
            if (e != cudaSuccess) return e;
            return launch_sketch_tc(n, r.d, A, lda, (const float *)h->omt.p, B, (float *)h->skp.p,
                                    h->skp.bytes / sizeof(float), 0, n, (int *)h->status.p, s);
        }
    }
    return launch_sketch<T, T>(n, r.d, A, lda, om, B, (T *)h->skp.p, h->skp.bytes / sizeof(T), s);
}

template <typename T>
rcp_status factor_impl(rcp_handle *h, int n, T *A, int lda, double *Dd, double *Ds, int *perm, const Resolved &r,
                       cudaStream_t s, rcp_stats *stats, bool presketched = false) {
    RCP_TRY(ensure_factor_ws<T>(h, n, r));
    FactorWork<T> w = make_work<T>(h, n, A, lda, Dd, Ds, perm, r);
    CU_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(int), s));
    CU_TRY(cudaMemsetAsync(h->bar.p, 0, sizeof(unsigned), s));
    CU_TRY(cudaMemsetAsync(h->keys.p, 0, PANEL_KEY_WORDS * sizeof(unsigned long long), s));
    CU_TRY(launch_factor_init<T>(w, s));
    const T *om = (const T *)r.omega;
    if (!presketched) {   // (else Omega and B = Omega A were formed while A arrived)
        PhaseScope ps(h, s, PH_SKETCH);
        if (!om) {
            CU_TRY(launch_omega<T>(r.d, n, r.seed, (T *)h->om.p, s));
            om = (const T *)h->om.p;
        }
        CU_TRY(sketch_for<T>(h, r, n, A, lda, om, w.B, s));
    }
    const int nblk = (n + r.b - 1) / r.b;
    int npanels = nblk;
    if (r.guard_r > 0) {
        // Algorithm 2: its decisions change where panels end, so the host reads the state after
        // every block; a request either recomputes the sketch of the Schur complement (a fresh
        // Omega' from Philox stream = recomputation number, d x (n - k)) or stops the
        // factorization at k (the Schur complement counts as zero)
        auto set_int = [&](size_t off, int v) -> cudaError_t {
            return cudaMemcpyAsync((char *)h->state.p + off, &v, sizeof v, cudaMemcpyHostToDevice, s);
        };
        const int maxpan = nblk + r.guard_r;
        int blk = 0, k0h = 0;
        while (k0h < n) {
            if (blk >= maxpan) return RCP_ECUDA;   // cannot happen: each request ends one panel early
            {
                PhaseScope ps(h, s, PH_PANEL);
                CU_TRY(launch_panel<T>(w, s));
            }
            {
                PhaseScope ps(h, s, PH_INTERCHANGE);
                CU_TRY(launch_interchange<T>(w, s, true));   // the panel marked its moved indices
                CU_TRY(launch_panel_record<T>(w, blk, s));
            }
            {
                PhaseScope ps(h, s, PH_TRAILING);
                CU_TRY(launch_trailing<T>(w, k0h, (int)r.prec, s));   // the panel ends at or after k0h
            }
            ++blk;
            FactorState st;
            int bits = 0;
            CU_TRY(cudaMemcpyAsync(&st, h->state.p, sizeof st, cudaMemcpyDeviceToHost, s));
            CU_TRY(cudaMemcpyAsync(&bits, h->status.p, sizeof bits, cudaMemcpyDeviceToHost, s));
            CU_TRY(cudaStreamSynchronize(s));
            if (bits) break;
            if (st.guard_req == 1) {
                const int k = st.guard_k, m = n - k, q = st.nresk + 1;
                PhaseScope ps(h, s, PH_SKETCH);
                CU_TRY(launch_omega<T>(r.d, m, r.seed, (T *)h->om.p, s, (uint64_t)q));
                CU_TRY(sketch_for<T>(h, r, m, A + (size_t)k + (size_t)k * lda, lda, (const T *)h->om.p,
                                     w.B + (size_t)k * r.d, s));
                CU_TRY(set_int(offsetof(FactorState, nresk), q));
                CU_TRY(set_int(offsetof(FactorState, guard_req), 0));
            } else if (st.guard_req == 2) {
                const int k = st.guard_k;
                CU_TRY(launch_guard_zero<T>(n, k, A, lda, Dd, Ds, s));
                CU_TRY(set_int(offsetof(FactorState, rank), k));
                CU_TRY(set_int(offsetof(FactorState, next), n));
                if (st.info == 0) CU_TRY(set_int(offsetof(FactorState, info), k + 1));
                CU_TRY(set_int(offsetof(FactorState, guard_req), 0));
                break;
            }
            k0h = st.next;
        }
        npanels = blk;
    }
    for (int blk = 0; blk < (r.guard_r > 0 ? 0 : nblk); ++blk) {
        if (r.qb) {
            // q = b: the block's candidates from a partial QRCP of the sketch, interchanged to
            // the first positions of the block before the panel
            PhaseScope ps(h, s, PH_SKETCH);
            CU_TRY(launch_qrcp<T>(w, r.b, s));
            CU_TRY(launch_interchange<T>(w, s));
        }
        {
            PhaseScope ps(h, s, PH_PANEL);
            CU_TRY(launch_panel<T>(w, s));
        }
        {
            PhaseScope ps(h, s, PH_INTERCHANGE);
            CU_TRY(launch_interchange<T>(w, s, true));   // the panel marked its moved indices
            CU_TRY(launch_panel_record<T>(w, blk, s));
        }
        {
            PhaseScope ps(h, s, PH_TRAILING);
            CU_TRY(launch_trailing<T>(w, std::min(n, (blk + 1) * r.b), (int)r.prec, s));
        }
        if (r.qb) {
            PhaseScope ps(h, s, PH_SKETCH);
            if constexpr (std::is_same<T, float>::value) {
                if (tc_prec(r.prec)) CU_TRY(launch_block_sketch_update_tc(w, w.tmpL, (float *)h->omt.p, s));
                else CU_TRY(launch_block_sketch_update<T>(w, w.tmpL, s));
            } else {
                CU_TRY(launch_block_sketch_update<T>(w, w.tmpL, s));
            }
        }
    }
    {
        PhaseScope ps(h, s, PH_INTERCHANGE);
        CU_TRY(launch_lrows_permute<T>(w, npanels, s));
    }
    CU_TRY(launch_factor_finish<T>(w, s));
    if (!stats) return RCP_OK;
    CU_TRY(cudaStreamSynchronize(s));
    FactorState st;
    int bits = 0;
    CU_TRY(cudaMemcpy(&st, h->state.p, sizeof st, cudaMemcpyDeviceToHost));
    CU_TRY(cudaMemcpy(&bits, h->status.p, sizeof bits, cudaMemcpyDeviceToHost));
    double maxA = bits_to_double(st.maxA_bits);
    stats->growth_D = maxA > 0.0 ? bits_to_double(st.maxD_bits) / maxA : 0.0;
    stats->max_abs_L = bits_to_double(st.maxL_bits);
    stats->min_sketch_ratio = st.min_ratio;
    stats->n_2x2 = st.n2x2;
    stats->info = st.info;
    stats->device_flags = bits;
    stats->rank = st.rank;
    stats->resketches = st.nresk;
    rcp_status e = status_from_bits(bits);
    if (e != RCP_OK) return e;
    return st.info > 0 ? (rcp_status)st.info : RCP_OK;
}

int solve_nb(int n) { return (n + 63) / 64; }

// Workspace of the solves (work area and flags) for n x nrhs.
// The solves' readers take a block as done when its flag (FP64) or its 64-bit words (FP32, the
// value with the epoch in the high half) carry the current epoch.  The epoch is chosen on the host,
// so a call replayed from a CUDA graph runs with the epoch of its capture and would find its own
// previous replay's flags and words already "current": the flags and, for FP32 factors, the word
// arrays are cleared on the stream before every solve (a few microseconds), which also removes
// any doubles an FP64 solve left where FP32 words are read.
template <typename T>
rcp_status prepare_solve_ws(rcp_handle *h, int n, int nrhs, cudaStream_t s) {
    RCP_TRY(ensure_small(h));
    RCP_TRY(grow_zeroed(h->Y, solve_work_bytes<T>(n, nrhs), s, false));
    const int nb = solve_nb(n);
    RCP_TRY(grow(h->flags, (size_t)(2 * nb + 2) * sizeof(int)));
    CU_TRY(cudaMemsetAsync(h->flags.p, 0, (size_t)(2 * nb) * sizeof(int), s));
    if (sizeof(T) == sizeof(float))
        CU_TRY(cudaMemsetAsync(h->Y.p, 0, 2 * (size_t)n * nrhs * sizeof(unsigned long long), s));
    return RCP_OK;
}

// reuse_inv: a later solve of the same refinement (same factor, n and nrhs, workspace untouched
// since): the inverted diagonal blocks of the first solve are used again.
template <typename T>
rcp_status solve_impl(rcp_handle *h, int n, int nrhs, const T *L, int lda, const double *Dd, const double *Ds,
                      const int *perm, double *X, int ldx, const int *skip, cudaStream_t s, bool reuse_inv = false) {
    const void *y0 = h->Y.p;
    const size_t y0b = h->Y.bytes;
    RCP_TRY(prepare_solve_ws<T>(h, n, nrhs, s));
    if (h->Y.p != y0 || h->Y.bytes != y0b) reuse_inv = false;   // the workspace was reallocated
    PhaseScope ps(h, s, PH_SOLVE);
    CU_TRY(launch_solve<T>(n, nrhs, L, lda, Dd, Ds, perm, X, ldx, (T *)h->Y.p, (int *)h->flags.p,
                           (int *)h->status.p, skip, s, reuse_inv));
    return RCP_OK;
}

bool valid_prec(rcp_prec p) { return p >= RCP_FP64 && p <= RCP_F16X3; }

// ||L||_1 exactly and ||L^{-1}||_1 by Higham's estimator ("FORTRAN codes for estimating the
// one-norm of a real or complex matrix", ACM TOMS 14 (1988), Algorithm 4.1, after Hager, 1984):
// a few products with L^{-1} and L^{-T} steer a unit vector towards a column of L^{-1} of
// largest 1-norm; every value it returns is ||L^{-1} x||_1 / ||x||_1 for some x, a lower bound.
template <typename T>
rcp_status l_norms_impl(rcp_handle *h, int n, const T *L, int lda, cudaStream_t s, double *nL, double *nLinv) {
    RCP_TRY(prepare_solve_ws<T>(h, n, 1, s));
    RCP_TRY(grow(h->iperm, (size_t)n * sizeof(int)));
    RCP_TRY(grow(h->gmZ, (size_t)n * sizeof(double)));
    CU_TRY(launch_iota(n, (int *)h->iperm.p, s));
    RefineScalars *sc = (RefineScalars *)h->scal.p;
    CU_TRY(launch_l_norm1<T>(n, L, lda, &sc->mx[0], s));
    unsigned long long bits = 0;
    CU_TRY(cudaMemcpyAsync(&bits, &sc->mx[0], sizeof bits, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    *nL = bits_to_double(bits);
    double *dv = (double *)h->gmZ.p;
    std::vector<double> x((size_t)n), y((size_t)n), xi((size_t)n), z((size_t)n);
    // v <- L^{-1} v (mode 0) or L^{-T} v (mode 1) through the device
    auto apply = [&](int mode, const std::vector<double> &in, std::vector<double> &out) -> rcp_status {
        CU_TRY(cudaMemcpyAsync(dv, in.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CU_TRY(launch_tri_solve<T>(n, L, lda, (const int *)h->iperm.p, dv, (T *)h->Y.p, (int *)h->flags.p,
                                   (int *)h->status.p, mode, s));
        CU_TRY(cudaMemcpyAsync(out.data(), dv, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        int st = 0;
        CU_TRY(cudaMemcpy(&st, h->status.p, sizeof st, cudaMemcpyDeviceToHost));
        return st ? status_from_bits(st) : RCP_OK;
    };
    auto norm1 = [&](const std::vector<double> &v) { double t = 0.0; for (double a : v) t += std::fabs(a); return t; };
    auto amax = [&](const std::vector<double> &v) {
        int j = 0;
        for (int i = 1; i < n; ++i) if (std::fabs(v[i]) > std::fabs(v[j])) j = i;
        return j;
    };
    for (int i = 0; i < n; ++i) x[i] = 1.0 / n;
    RCP_TRY(apply(0, x, y));
    double est = norm1(y);
    if (n > 1) {
        for (int i = 0; i < n; ++i) xi[i] = y[i] >= 0.0 ? 1.0 : -1.0;
        RCP_TRY(apply(1, xi, z));
        int j = amax(z);
        for (int iter = 2; iter <= 5; ++iter) {
            std::fill(x.begin(), x.end(), 0.0);
            x[j] = 1.0;
            RCP_TRY(apply(0, x, y));
            const double old = est;
            est = norm1(y);
            bool same = true;
            for (int i = 0; i < n && same; ++i) same = (y[i] >= 0.0 ? 1.0 : -1.0) == xi[i];
            if (same || est <= old) { est = std::max(est, old); break; }
            for (int i = 0; i < n; ++i) xi[i] = y[i] >= 0.0 ? 1.0 : -1.0;
            RCP_TRY(apply(1, xi, z));
            const int jlast = j;
            j = amax(z);
            if (std::fabs(z[jlast]) == std::fabs(z[j])) break;   // no column promises more
        }
        // the alternative vector x_i = (-1)^i (1 + i / (n - 1)), ||x||_1 = 3n/2
        for (int i = 0; i < n; ++i) x[i] = (i % 2 ? -1.0 : 1.0) * (1.0 + (double)i / (n - 1));
        RCP_TRY(apply(0, x, y));
        est = std::max(est, 2.0 * norm1(y) / (3.0 * n));
    }
    *nLinv = est;
    return RCP_OK;
}

}  // namespace

extern "C" {

rcp_status rcp_create(rcp_handle **h) {
    if (!h) return RCP_EINVAL;
    *h = new (std::nothrow) rcp_handle();
    if (!*h) return RCP_ENOMEM;
    cudaGetDevice(&(*h)->device);
    return RCP_OK;
}

void rcp_destroy(rcp_handle *h) {
    if (!h) return;
    Buf *all[] = {&h->psnap, &h->pinv, &h->pbounds, &h->bord, &h->bom, &h->bticket, &h->bscr, &h->tcops, &h->keys, &h->skp, &h->omt, &h->trace, &h->status, &h->state, &h->bar, &h->scal, &h->om, &h->B, &h->Wbuf, &h->Lc, &h->Lg, &h->lpos, &h->moved,
                  &h->s1v, &h->s2v, &h->s3v, &h->s1i, &h->s2i, &h->pay, &h->tmpA, &h->tmpL, &h->tmpP, &h->Y, &h->flags,
                  &h->R, &h->Dc, &h->part, &h->A64, &h->F, &h->Bh, &h->Xh, &h->Dd, &h->Ds, &h->perm,
                  &h->gmV, &h->gmZ, &h->gmP, &h->gmH, &h->iperm};
    for (Buf *b : all)
        if (b->p) cudaFree(b->p);
    for (auto &e : h->events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (auto e : h->pool) cudaEventDestroy(e);
    for (auto e : h->copy_events) cudaEventDestroy(e);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    delete h;
}

const char *rcp_status_string(int s) {
    switch (s) {
        case RCP_OK: return "ok";
        case RCP_EINVAL: return "invalid argument";
        case RCP_ENOMEM: return "device allocation failed";
        case RCP_ECUDA: return "CUDA runtime error";
        case RCP_ENONFINITE: return "non-finite value met during the factorization";
        case RCP_ETIMEOUT: return "a bounded device-side wait ran out";
        case RCP_ENOCONV: return "refinement did not reach the tolerance";
        case RCP_EUNSUPPORTED: return "unsupported size or option";
        default: return s > 0 ? "zero pivot (info > 0)" : "unknown status";
    }
}

rcp_status rcp_sync(rcp_handle *h, rcp_stream_t stream) {
    if (!h) return RCP_EINVAL;
    CU_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (!h->status.p) return RCP_OK;
    int bits = 0;
    CU_TRY(cudaMemcpy(&bits, h->status.p, sizeof bits, cudaMemcpyDeviceToHost));
    return status_from_bits(bits);
}

rcp_status rcp_reserve(rcp_handle *h, int n, int nrhs, const rcp_opts *opts) {
    if (!h || n < 0 || nrhs < 0) return RCP_EINVAL;
    Resolved r;
    RCP_TRY(resolve(n, opts, r, h->spec_mode));
    if (r.prec == RCP_FP64) RCP_TRY(ensure_factor_ws<double>(h, n, r));
    else RCP_TRY(ensure_factor_ws<float>(h, n, r));
    RCP_TRY(grow_zeroed(h->Y,
                        r.prec == RCP_FP64 ? solve_work_bytes<double>(n, std::max(nrhs, 1))
                                           : solve_work_bytes<float>(n, std::max(nrhs, 1)),
                        nullptr, true));
    RCP_TRY(grow(h->R, (size_t)n * std::max(nrhs, 1) * sizeof(double)));
    RCP_TRY(grow(h->Dc, (size_t)n * std::max(nrhs, 1) * sizeof(double)));
    RCP_TRY(grow(h->part, symv_part_doubles(n, std::max(nrhs, 1)) * sizeof(double)));
    return RCP_OK;
}

rcp_status rcp_factor(rcp_handle *h, int n, void *A, int lda, double *Dd, double *Ds, int *perm, const rcp_opts *opts,
                      rcp_stream_t stream, rcp_stats *stats) {
    if (!h || n < 0 || (n > 0 && (!A || !Dd || !Ds || !perm)) || lda < (n > 0 ? n : 1)) return RCP_EINVAL;
    if (stats) std::memset(stats, 0, sizeof *stats);
    if (n == 0) return RCP_OK;
    Resolved r;
    RCP_TRY(resolve(n, opts, r, h->spec_mode));
    cudaStream_t s = (cudaStream_t)stream;
    if (r.prec == RCP_FP64) return factor_impl<double>(h, n, (double *)A, lda, Dd, Ds, perm, r, s, stats);
    return factor_impl<float>(h, n, (float *)A, lda, Dd, Ds, perm, r, s, stats);
}

rcp_status rcp_solve(rcp_handle *h, int n, int nrhs, const void *LA, int lda, const double *Dd, const double *Ds,
                     const int *perm, rcp_prec prec, double *X, int ldx, rcp_stream_t stream) {
    if (!h || n < 0 || nrhs < 0 || !valid_prec(prec)) return RCP_EINVAL;
    if (n == 0 || nrhs == 0) return RCP_OK;
    if (!LA || !Dd || !Ds || !perm || !X || lda < n || ldx < n) return RCP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == RCP_FP64) return solve_impl<double>(h, n, nrhs, (const double *)LA, lda, Dd, Ds, perm, X, ldx, nullptr, s);
    return solve_impl<float>(h, n, nrhs, (const float *)LA, lda, Dd, Ds, perm, X, ldx, nullptr, s);
}

// host_checks: the caller synchronizes at the end anyway (it fills host statistics), so after each
// iteration's convergence check the host reads the flag and stops launching: the iterations
// after convergence are not launched at all (they would only skip their work on the device, at
// the cost of their launches: ~0.4 ms for eight of them at n = 16384).  Without it (no host
// statistics, e.g. inside a graph capture) all max_iter iterations are launched and skip.
static rcp_status refine_run(rcp_handle *h, int n, int nrhs, const double *A64, int lda, const void *LA, int ldla,
                             const double *Dd, const double *Ds, const int *perm, rcp_prec prec, const double *Bv,
                             int ldb, double *X, int ldx, double tol, int max_iter, rcp_stream_t stream,
                             rcp_stats *stats, bool host_checks);

rcp_status rcp_refine(rcp_handle *h, int n, int nrhs, const double *A64, int lda, const void *LA, int ldla,
                      const double *Dd, const double *Ds, const int *perm, rcp_prec prec, const double *Bv, int ldb,
                      double *X, int ldx, double tol, int max_iter, rcp_stream_t stream, rcp_stats *stats) {
    return refine_run(h, n, nrhs, A64, lda, LA, ldla, Dd, Ds, perm, prec, Bv, ldb, X, ldx, tol, max_iter, stream, stats,
                      stats != nullptr);
}

static rcp_status refine_run(rcp_handle *h, int n, int nrhs, const double *A64, int lda, const void *LA, int ldla,
                             const double *Dd, const double *Ds, const int *perm, rcp_prec prec, const double *Bv,
                             int ldb, double *X, int ldx, double tol, int max_iter, rcp_stream_t stream,
                             rcp_stats *stats, bool host_checks) {
    if (!h || n < 0 || nrhs < 0 || nrhs > kMaxRhs || !valid_prec(prec) || max_iter < 0) return RCP_EINVAL;
    if (stats) std::memset(stats, 0, sizeof *stats);
    if (n == 0 || nrhs == 0) return RCP_OK;
    if (!A64 || !LA || !Dd || !Ds || !perm || !Bv || !X || lda < n || ldla < n || ldb < n || ldx < n) return RCP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    RCP_TRY(ensure_small(h));
    RCP_TRY(grow(h->R, (size_t)n * nrhs * sizeof(double)));
    RCP_TRY(grow(h->Dc, (size_t)n * nrhs * sizeof(double)));
    RCP_TRY(grow(h->part, symv_part_doubles(n, nrhs) * sizeof(double)));
    RefineScalars *sc = (RefineScalars *)h->scal.p;
    double *R = (double *)h->R.p, *Dc = (double *)h->Dc.p, *part = (double *)h->part.p;
    CU_TRY(cudaMemsetAsync(sc, 0, offsetof(RefineScalars, berr), s));
    CU_TRY(launch_anorm(n, A64, lda, part, &sc->anorm, s));
    CU_TRY(cudaMemcpy2DAsync(X, (size_t)ldx * sizeof(double), Bv, (size_t)ldb * sizeof(double), (size_t)n * sizeof(double),
                             nrhs, cudaMemcpyDeviceToDevice, s));
    // the corrections' solves reuse the first solve's inverted diagonal blocks (same factor)
    auto do_solve = [&](double *rhs, const int *skip, bool reuse) -> rcp_status {
        if (prec == RCP_FP64)
            return solve_impl<double>(h, n, nrhs, (const double *)LA, ldla, Dd, Ds, perm, rhs, rhs == X ? ldx : n, skip, s,
                                      reuse);
        return solve_impl<float>(h, n, nrhs, (const float *)LA, ldla, Dd, Ds, perm, rhs, rhs == X ? ldx : n, skip, s,
                                 reuse);
    };
    RCP_TRY(do_solve(X, nullptr, false));
    for (int it = 0; it <= max_iter; ++it) {
        {
            PhaseScope ps(h, s, PH_RESIDUAL);
            CU_TRY(launch_symv_residual(n, nrhs, A64, lda, X, ldx, Bv, ldb, R, n, part, sc->mx, &sc->conv, s));
        }
        CU_TRY(launch_refine_check(nrhs, sc->mx, &sc->anorm, tol, &sc->conv, &sc->berr, &sc->prev, &sc->iters,
                                   it < max_iter, s));
        if (it == max_iter) break;
        if (host_checks) {
            int conv = 0;
            CU_TRY(cudaMemcpyAsync(&conv, &sc->conv, sizeof conv, cudaMemcpyDeviceToHost, s));
            CU_TRY(cudaStreamSynchronize(s));
            if (conv != 0) break;
        }
        CU_TRY(cudaMemcpyAsync(Dc, R, (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RCP_TRY(do_solve(Dc, &sc->conv, true));
        CU_TRY(launch_axpy_update(n, nrhs, X, ldx, Dc, n, &sc->conv, s));
    }
    if (!stats) return RCP_OK;
    CU_TRY(cudaStreamSynchronize(s));
    RefineScalars host;
    CU_TRY(cudaMemcpy(&host, sc, offsetof(RefineScalars, mx), cudaMemcpyDeviceToHost));
    int bits = 0;
    CU_TRY(cudaMemcpy(&bits, h->status.p, sizeof bits, cudaMemcpyDeviceToHost));
    stats->berr = host.berr;
    stats->anorm = host.anorm;
    stats->refine_iters = host.iters;
    stats->device_flags = bits;
    rcp_status e = status_from_bits(bits);
    if (e != RCP_OK) return e;
    if (!(host.berr <= tol)) return RCP_ENOCONV;
    return RCP_OK;
}

// Least-squares problem of GMRES: min_y || beta e_1 - H y ||_2 with H the (k+1) x k upper
// Hessenberg matrix of the Arnoldi process, by Givens rotations (Saad and Schultz, 1986).
rcp_status rcp_gmres_lsq(int k, const double *H, int ldh, double beta, double *y, double *resid) {
    if (k < 0 || !resid || (k > 0 && (!H || !y || ldh < k + 1))) return RCP_EINVAL;
    std::vector<double> R((size_t)(k + 1) * (k > 0 ? k : 1)), g((size_t)k + 1, 0.0);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i <= k; ++i) R[(size_t)i + (size_t)j * (k + 1)] = i <= j + 1 ? H[(size_t)i + (size_t)j * ldh] : 0.0;
    g[0] = beta;
    auto at = [&](int i, int j) -> double & { return R[(size_t)i + (size_t)j * (k + 1)]; };
    for (int j = 0; j < k; ++j) {
        // the rotation that zeroes H(j+1, j) against H(j, j), applied to rows j, j+1
        const double a = at(j, j), b = at(j + 1, j), r = std::hypot(a, b);
        const double c = r > 0.0 ? a / r : 1.0, sn = r > 0.0 ? b / r : 0.0;
        for (int l = j; l < k; ++l) {
            const double t1 = at(j, l), t2 = at(j + 1, l);
            at(j, l) = c * t1 + sn * t2;
            at(j + 1, l) = -sn * t1 + c * t2;
        }
        const double t1 = g[j], t2 = g[j + 1];
        g[j] = c * t1 + sn * t2;
        g[j + 1] = -sn * t1 + c * t2;
    }
    *resid = std::fabs(g[k]);
    for (int j = k - 1; j >= 0; --j) {
        double t = g[j];
        for (int l = j + 1; l < k; ++l) t -= at(j, l) * y[l];
        y[j] = at(j, j) != 0.0 ? t / at(j, j) : 0.0;   // a zero pivot: exact breakdown of a singular H
    }
    return RCP_OK;
}

namespace {
constexpr int kGmresMaxRestart = 128;
constexpr double kGmresInnerTol = 1e-10;   // relative reduction of the preconditioned residual per cycle
}

rcp_status rcp_refine_gmres(rcp_handle *h, int n, int nrhs, const double *A64, int lda, const void *LA, int ldla,
                            const double *Dd, const double *Ds, const int *perm, rcp_prec prec, const double *Bv,
                            int ldb, double *X, int ldx, double tol, int max_outer, int restart, int use_x,
                            rcp_stream_t stream, rcp_stats *stats) {
    if (!h || n < 0 || nrhs < 0 || nrhs > kMaxRhs || !valid_prec(prec) || max_outer < 0) return RCP_EINVAL;
    if (restart <= 0) restart = 64;
    if (restart > kGmresMaxRestart) return RCP_EINVAL;
    if (stats) std::memset(stats, 0, sizeof *stats);
    if (n == 0 || nrhs == 0) return RCP_OK;
    if (!A64 || !LA || !Dd || !Ds || !perm || !Bv || !X || lda < n || ldla < n || ldb < n || ldx < n) return RCP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int m = restart;
    RCP_TRY(ensure_small(h));
    RCP_TRY(grow(h->R, (size_t)n * sizeof(double)));
    RCP_TRY(grow(h->part, symv_part_doubles(n, 1) * sizeof(double)));
    RCP_TRY(grow(h->gmV, (size_t)n * (m + 1) * sizeof(double)));
    RCP_TRY(grow(h->gmZ, (size_t)n * sizeof(double)));
    RCP_TRY(grow(h->gmP, gm_part_doubles(n, m + 1) * sizeof(double)));
    RCP_TRY(grow(h->gmH, (size_t)(2 * (m + 1) + 2) * sizeof(double)));
    RefineScalars *sc = (RefineScalars *)h->scal.p;
    double *R = (double *)h->R.p, *part = (double *)h->part.p, *V = (double *)h->gmV.p, *Z = (double *)h->gmZ.p;
    double *gp = (double *)h->gmP.p, *hd = (double *)h->gmH.p;
    double *h1 = hd, *h2 = hd + (m + 1), *nrm2 = hd + 2 * (m + 1);
    CU_TRY(cudaMemsetAsync(Z, 0, (size_t)n * sizeof(double), s));
    CU_TRY(launch_anorm(n, A64, lda, part, &sc->anorm, s));
    auto solve1 = [&](double *v, int ld, int cols) -> rcp_status {
        if (prec == RCP_FP64) return solve_impl<double>(h, n, cols, (const double *)LA, ldla, Dd, Ds, perm, v, ld, nullptr, s);
        return solve_impl<float>(h, n, cols, (const float *)LA, ldla, Dd, Ds, perm, v, ld, nullptr, s);
    };
    if (!use_x) {
        CU_TRY(cudaMemcpy2DAsync(X, (size_t)ldx * sizeof(double), Bv, (size_t)ldb * sizeof(double),
                                 (size_t)n * sizeof(double), nrhs, cudaMemcpyDeviceToDevice, s));
        RCP_TRY(solve1(X, ldx, nrhs));
    }
    double anorm = 0.0;
    CU_TRY(cudaMemcpyAsync(&anorm, &sc->anorm, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    std::vector<double> H((size_t)(m + 1) * m), y((size_t)m), hh((size_t)2 * (m + 1) + 1);
    int outer_total = 0, inner_total = 0;
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        double *x = X + (size_t)c * ldx;
        const double *b = Bv + (size_t)c * ldb;
        double berr = INFINITY;
        for (int outer = 0;; ++outer) {
            // r = b - A x (FP64) and its backward error
            {
                PhaseScope ps(h, s, PH_RESIDUAL);
                CU_TRY(launch_symv_residual(n, 1, A64, lda, x, ldx, b, ldb, R, n, part, sc->mx, nullptr, s));
            }
            unsigned long long mxh[2];
            CU_TRY(cudaMemcpyAsync(mxh, sc->mx, sizeof mxh, cudaMemcpyDeviceToHost, s));
            CU_TRY(cudaStreamSynchronize(s));
            double rm, xm;
            std::memcpy(&rm, &mxh[0], sizeof rm);
            std::memcpy(&xm, &mxh[1], sizeof xm);
            berr = (anorm > 0.0 && xm > 0.0) ? rm / (anorm * xm) : (rm > 0.0 ? INFINITY : 0.0);
            if (!std::isfinite(berr) && outer > 0) return RCP_ENONFINITE;
            if (berr <= tol || outer == max_outer) break;
            // one GMRES cycle on M^{-1} A d = M^{-1} r: v_0 = M^{-1} r / beta
            CU_TRY(cudaMemcpyAsync(V, R, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            RCP_TRY(solve1(V, n, 1));
            CU_TRY(launch_gm_dots(n, 1, V, n, V, gp, nrm2, s));
            double b2 = 0.0;
            CU_TRY(cudaMemcpyAsync(&b2, nrm2, sizeof b2, cudaMemcpyDeviceToHost, s));
            CU_TRY(cudaStreamSynchronize(s));
            if (!std::isfinite(b2)) return RCP_ENONFINITE;
            if (!(b2 > 0.0)) break;   // M^{-1} r = 0: nothing left to correct
            const double beta = std::sqrt(b2);
            CU_TRY(launch_gm_scale(n, 1.0 / beta, V, s));
            int k = 0;
            double res = beta;
            for (int j = 0; j < m; ++j) {
                double *vj = V + (size_t)j * n, *u = V + (size_t)(j + 1) * n;
                // u = -M^{-1} A v_j (the residual kernel with a zero right-hand side gives -A v_j)
                {
                    PhaseScope ps(h, s, PH_RESIDUAL);
                    CU_TRY(launch_symv_residual(n, 1, A64, lda, vj, n, Z, n, u, n, part, sc->mx, nullptr, s));
                }
                RCP_TRY(solve1(u, n, 1));
                // classical Gram-Schmidt, twice, against v_0 .. v_j; then ||u||^2
                CU_TRY(launch_gm_dots(n, j + 1, V, n, u, gp, h1, s));
                CU_TRY(launch_gm_update(n, j + 1, V, n, h1, -1.0, u, s));
                CU_TRY(launch_gm_dots(n, j + 1, V, n, u, gp, h2, s));
                CU_TRY(launch_gm_update(n, j + 1, V, n, h2, -1.0, u, s));
                CU_TRY(launch_gm_dots(n, 1, u, n, u, gp, nrm2, s));
                CU_TRY(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost, s));
                CU_TRY(cudaStreamSynchronize(s));
                // u held -M^{-1} A v_j: H(i, j) = -(h1 + h2)_i, and v_{j+1} = -u / ||u||
                for (int i = 0; i <= j; ++i) H[(size_t)i + (size_t)j * (m + 1)] = -(hh[i] + hh[(size_t)(m + 1) + i]);
                const double un2 = hh[(size_t)2 * (m + 1)];
                if (!std::isfinite(un2)) return RCP_ENONFINITE;
                const double hn = std::sqrt(un2);
                H[(size_t)(j + 1) + (size_t)j * (m + 1)] = hn;
                k = j + 1;
                ++inner_total;
                RCP_TRY(rcp_gmres_lsq(k, H.data(), m + 1, beta, y.data(), &res));
                if (!(hn > 0.0) || res <= kGmresInnerTol * beta) break;   // breakdown (exact) or converged
                CU_TRY(launch_gm_scale(n, -1.0 / hn, u, s));
            }
            // x += V_k y
            CU_TRY(cudaMemcpyAsync(h1, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
            CU_TRY(launch_gm_update(n, k, V, n, h1, 1.0, x, s));
            ++outer_total;
        }
        if (!(berr <= worst)) worst = berr;
    }
    CU_TRY(cudaStreamSynchronize(s));
    int bits = 0;
    CU_TRY(cudaMemcpy(&bits, h->status.p, sizeof bits, cudaMemcpyDeviceToHost));
    if (stats) {
        stats->berr = worst;
        stats->anorm = anorm;
        stats->refine_iters = outer_total;
        stats->gmres_iters = inner_total;
        stats->device_flags = bits;
    }
    rcp_status e = status_from_bits(bits);
    if (e != RCP_OK) return e;
    if (!(worst <= tol)) return RCP_ENOCONV;
    return RCP_OK;
}

rcp_status rcp_sysv(rcp_handle *h, int n, int nrhs, const double *A64, int lda, const double *Bv, int ldb, double *X,
                    int ldx, const rcp_opts *opts, double tol, int max_iter, int host_buffers, rcp_stream_t stream,
                    rcp_stats *stats) {
    if (!h || !stats || n < 0 || nrhs < 0 || nrhs > kMaxRhs || max_iter < 0) return RCP_EINVAL;
    std::memset(stats, 0, sizeof *stats);
    if (n == 0 || nrhs == 0) return RCP_OK;
    if (!A64 || !Bv || !X || lda < n || ldb < n || ldx < n) return RCP_EINVAL;
    Resolved r;
    RCP_TRY(resolve(n, opts, r, h->spec_mode));
    cudaStream_t s = (cudaStream_t)stream;
    RCP_TRY(ensure_small(h));
    const double *dA = A64, *dB = Bv;
    double *dX = X;
    int dlda = lda, dldb = ldb, dldx = ldx;
    const bool f64 = r.prec == RCP_FP64;
    RCP_TRY(grow(h->F, (size_t)n * n * (f64 ? sizeof(double) : sizeof(float))));
    RCP_TRY(grow(h->Dd, (size_t)n * sizeof(double)));
    RCP_TRY(grow(h->Ds, (size_t)n * sizeof(double)));
    RCP_TRY(grow(h->perm, (size_t)n * sizeof(int)));
    bool presketched = false;
    if (host_buffers) {
        RCP_TRY(grow(h->A64, (size_t)n * n * sizeof(double)));
        RCP_TRY(grow(h->Bh, (size_t)n * nrhs * sizeof(double)));
        RCP_TRY(grow(h->Xh, (size_t)n * nrhs * sizeof(double)));
        dA = (const double *)h->A64.p; dB = (const double *)h->Bh.p; dX = (double *)h->Xh.p;
        dlda = dldb = dldx = n;
        const int nblk = (n + kHostCopyCols - 1) / kHostCopyCols;
        // FP32 factors: the blocks of A are copied on a second stream, and as each lands its
        // columns are rounded to FP32 and its columns of B = Omega A formed (they read only this
        // block and the rows of earlier ones), so the copy hides that work
        const bool overlap = !f64;
        if (overlap) {
            if (!h->copy_stream) CU_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
            while ((int)h->copy_events.size() < nblk + 1) {
                cudaEvent_t e;
                CU_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                h->copy_events.push_back(e);
            }
            RCP_TRY(ensure_factor_ws<float>(h, n, r));
            // the copies may start once the call's earlier work on s is done with the buffers
            CU_TRY(cudaEventRecord(h->copy_events[nblk], s));
            CU_TRY(cudaStreamWaitEvent(h->copy_stream, h->copy_events[nblk], 0));
        }
        cudaStream_t cs = overlap ? h->copy_stream : s;
        cudaEvent_t h2d_a = nullptr;
        if (h->profiling) {
            h2d_a = take_event(h);
            CU_TRY(cudaEventRecord(h2d_a, cs));
        }
        // only the lower triangle is read: copy it as rectangles of kHostCopyCols columns from
        // each block's diagonal down (half the bytes of the full matrix)
        for (int b = 0; b < nblk; ++b) {
            const int j0 = b * kHostCopyCols, wcols = std::min(kHostCopyCols, n - j0);
            CU_TRY(cudaMemcpy2DAsync((double *)h->A64.p + (size_t)j0 + (size_t)j0 * n, (size_t)n * sizeof(double),
                                     A64 + (size_t)j0 + (size_t)j0 * lda, (size_t)lda * sizeof(double),
                                     (size_t)(n - j0) * sizeof(double), wcols, cudaMemcpyHostToDevice, cs));
            if (overlap) CU_TRY(cudaEventRecord(h->copy_events[b], cs));
        }
        CU_TRY(cudaMemcpy2DAsync(h->Bh.p, (size_t)n * sizeof(double), Bv, (size_t)ldb * sizeof(double),
                                 (size_t)n * sizeof(double), nrhs, cudaMemcpyHostToDevice, cs));
        if (h2d_a) {
            cudaEvent_t h2d_b = take_event(h);
            CU_TRY(cudaEventRecord(h2d_b, cs));
            h->events.push_back({PH_H2D, h2d_a, h2d_b});
            h->launches[PH_H2D] += 1;
        }
        if (overlap) {
            const float *om = (const float *)r.omega;
            if (!om) {
                CU_TRY(launch_omega<float>(r.d, n, r.seed, (float *)h->om.p, s));
                om = (const float *)h->om.p;
            }
            if (tc_prec(r.prec)) CU_TRY(launch_omega_split(n, r.d, om, (float *)h->omt.p, s));
            for (int b = 0; b < nblk; ++b) {
                const int j0 = b * kHostCopyCols, j1 = std::min(n, j0 + kHostCopyCols);
                CU_TRY(cudaStreamWaitEvent(s, h->copy_events[b], 0));
                CU_TRY(launch_copy_lower_f64(n, dA, dlda, h->F.p, n, 1, s, j0, j1));
                if (tc_prec(r.prec))
                    CU_TRY(launch_sketch_tc(n, r.d, (const float *)h->F.p, n, (const float *)h->omt.p, (float *)h->B.p,
                                            (float *)h->skp.p, h->skp.bytes / sizeof(float), j0, j1,
                                            (int *)h->status.p, s));
                else
                    CU_TRY(launch_sketch_cols_f32(n, r.d, (const float *)h->F.p, n, om, (float *)h->B.p,
                                                  (float *)h->skp.p, h->skp.bytes / sizeof(float), j0, j1, s));
            }
            // the right-hand sides (last on the copy stream) before the refinement
            CU_TRY(cudaEventRecord(h->copy_events[nblk], cs));
            CU_TRY(cudaStreamWaitEvent(s, h->copy_events[nblk], 0));
            presketched = true;
        }
    }
    if (!presketched) CU_TRY(launch_copy_lower_f64(n, dA, dlda, h->F.p, n, f64 ? 0 : 1, s));
    rcp_stats fst;
    rcp_status fs;
    if (f64) fs = factor_impl<double>(h, n, (double *)h->F.p, n, (double *)h->Dd.p, (double *)h->Ds.p, (int *)h->perm.p, r, s, nullptr);
    else fs = factor_impl<float>(h, n, (float *)h->F.p, n, (double *)h->Dd.p, (double *)h->Ds.p, (int *)h->perm.p, r, s, nullptr,
                                 presketched);
    if (fs != RCP_OK) return fs;
    (void)fst;
    rcp_stats rst;
    rcp_status rs = refine_run(h, n, nrhs, dA, dlda, h->F.p, n, (double *)h->Dd.p, (double *)h->Ds.p, (int *)h->perm.p,
                               r.prec, dB, dldb, dX, dldx, tol, max_iter, stream, nullptr, true);
    if (rs != RCP_OK) return rs;
    // classic refinement stopped short of the tolerance (the factor is too inaccurate for this
    // system): GMRES-based refinement from the current iterate
    RefineScalars host;
    CU_TRY(cudaStreamSynchronize(s));
    CU_TRY(cudaMemcpy(&host, h->scal.p, offsetof(RefineScalars, mx), cudaMemcpyDeviceToHost));
    rcp_stats gst;
    std::memset(&gst, 0, sizeof gst);
    bool used_gmres = false;
    if (max_iter > 0 && !(host.berr <= tol)) {
        FactorState fs0;
        int bits0 = 0;
        CU_TRY(cudaMemcpy(&fs0, h->state.p, sizeof fs0, cudaMemcpyDeviceToHost));
        CU_TRY(cudaMemcpy(&bits0, h->status.p, sizeof bits0, cudaMemcpyDeviceToHost));
        if (bits0 == 0 && fs0.info == 0) {
            rcp_status gs = rcp_refine_gmres(h, n, nrhs, dA, dlda, h->F.p, n, (double *)h->Dd.p, (double *)h->Ds.p,
                                             (int *)h->perm.p, r.prec, dB, dldb, dX, dldx, tol, max_iter, 0, 1, stream,
                                             &gst);
            if (gs != RCP_OK && gs != RCP_ENOCONV) return gs;
            used_gmres = true;
        }
    }
    if (host_buffers)
        CU_TRY(cudaMemcpy2DAsync(X, (size_t)ldx * sizeof(double), dX, (size_t)n * sizeof(double), (size_t)n * sizeof(double),
                                 nrhs, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    // statistics of both phases
    FactorState st;
    int bits = 0;
    CU_TRY(cudaMemcpy(&st, h->state.p, sizeof st, cudaMemcpyDeviceToHost));
    CU_TRY(cudaMemcpy(&host, h->scal.p, offsetof(RefineScalars, mx), cudaMemcpyDeviceToHost));
    CU_TRY(cudaMemcpy(&bits, h->status.p, sizeof bits, cudaMemcpyDeviceToHost));
    double maxA = bits_to_double(st.maxA_bits);
    stats->growth_D = maxA > 0.0 ? bits_to_double(st.maxD_bits) / maxA : 0.0;
    stats->max_abs_L = bits_to_double(st.maxL_bits);
    stats->min_sketch_ratio = st.min_ratio;
    stats->n_2x2 = st.n2x2;
    stats->info = st.info;
    stats->device_flags = bits;
    stats->berr = used_gmres ? gst.berr : host.berr;
    stats->anorm = host.anorm;
    stats->refine_iters = host.iters + gst.refine_iters;
    stats->gmres_iters = gst.gmres_iters;
    stats->rank = st.rank;
    stats->resketches = st.nresk;
    (void)rst;
    const double berr_final = stats->berr;
    rcp_status e = status_from_bits(bits);
    if (e != RCP_OK) return e;
    if (st.info > 0) return (rcp_status)st.info;
    if (max_iter > 0 && !(berr_final <= tol)) return RCP_ENOCONV;
    return RCP_OK;
}

// ---- batched ragged systems ----

// order[batch] (largest systems first), then above[nmax + 1] (above[v]: systems with n > v)
static rcp_status batched_order(rcp_handle *h, int batch, int nmax, const int *n, cudaStream_t s) {
    RCP_TRY(grow(h->bord, ((size_t)batch + nmax + 1) * sizeof(int)));
    RCP_TRY(grow(h->bticket, 64));
    if (h->bord_n == n && h->bord_batch == batch && h->bord_nmax == nmax) return RCP_OK;
    // any permutation of the systems gives the same results; this one is for load balance
    CU_TRY(launch_batched_order(batch, nmax, n, (int *)h->bord.p, (int *)h->bord.p + batch, s));
    h->bord_n = n;
    h->bord_batch = batch;
    h->bord_nmax = nmax;
    return RCP_OK;
}

rcp_status rcp_factor_batched(rcp_handle *h, int batch, int nmax, const int *n, const double *const *A64,
                              const int *lda64, void *const *A, const int *lda, double *const *Dd,
                              double *const *Ds, int *const *perm, const rcp_opts *opts, int *info,
                              rcp_stream_t stream) {
    if (!h || batch < 0 || nmax < 0 || nmax > 65535) return RCP_EINVAL;
    if (batch == 0 || nmax == 0) return RCP_OK;
    if (!n || !A || !lda || !Dd || !Ds || !perm || !info || (A64 && !lda64)) return RCP_EINVAL;
    const rcp_prec prec = opts ? opts->prec : RCP_FP64;
    if (!valid_prec(prec)) return RCP_EINVAL;
    const bool f64 = prec == RCP_FP64;
    int b = (opts && opts->b > 0) ? opts->b : 32;
    const int dkey = (opts && opts->d > 0) ? opts->d : 0;
    int d = dkey > 0 ? dkey : std::min(b + 8, 128);
    int nt = 512, split = 0;   // CTA size; split > 0: systems with n <= split in a second launch
    if (!(opts && opts->b > 0))
        for (const auto &t : h->tuned)
            if (t.nmax == nmax && t.dkey == dkey && t.f64 == (int)f64) {   // the autotuned shape
                b = t.b; d = t.d; nt = t.nt; split = t.split;
            }
    if (h->bt_nt > 0 || h->bt_split > 0) {   // the schedule set on the handle
        nt = h->bt_nt > 0 ? h->bt_nt : 512;
        split = h->bt_split;
    }
    if (split >= nmax) split = 0;
    if (opts && opts->q_mode != 0 && opts->q_mode != 1) return RCP_EUNSUPPORTED;
    if (opts && opts->guard_r != 0) return RCP_EUNSUPPORTED;   // the safeguard is host-driven per system
    if (b > 512 || d > 128) return RCP_EUNSUPPORTED;
    const double alpha = (opts && opts->alpha > 0.0) ? opts->alpha : std::sqrt(2.0) / 2.0;
    if (!(alpha < 1.0)) return RCP_EINVAL;
    const size_t smem = f64 ? batched_factor_smem<double>(d, b, nmax) : batched_factor_smem<float>(d, b, nmax);
    if (smem > batched_max_smem()) return RCP_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    RCP_TRY(batched_order(h, batch, nmax, n, s));
    const void *om = opts ? opts->omega : nullptr;
    if (!om) {
        const uint64_t seed = opts ? opts->seed : 0;
        RCP_TRY(grow(h->bom, (size_t)d * nmax * (f64 ? sizeof(double) : sizeof(float))));
        if (h->bom_seed != seed || h->bom_d != d || h->bom_nmax != nmax || h->bom_f64 != (int)f64) {
            if (f64) CU_TRY(launch_omega<double>(d, nmax, seed, (double *)h->bom.p, s));
            else CU_TRY(launch_omega<float>(d, nmax, seed, (float *)h->bom.p, s));
            h->bom_seed = seed;
            h->bom_d = d;
            h->bom_nmax = nmax;
            h->bom_f64 = (int)f64;
        }
        om = h->bom.p;
    }
    // launches: {CTA size, order of the shared arrays, range of order[]}; with a split the systems
    // with n > split come first (512 threads), the others after (256 threads, arrays of order split)
    struct Leg { int nt, nm; const int *first, *last; int grid; };
    const int *above = (const int *)h->bord.p + batch;
    Leg legs[2];
    int nlegs = 0;
    if (split > 0) {
        legs[nlegs++] = {512, nmax, nullptr, above + split, 0};
        legs[nlegs++] = {256, split, above + split, nullptr, 0};
    } else {
        legs[nlegs++] = {nt, nmax, nullptr, nullptr, 0};
    }
    size_t scr = 0;
    for (int l = 0; l < nlegs; ++l) {
        Leg &g = legs[l];
        const size_t sm = f64 ? batched_factor_smem<double>(d, b, g.nm) : batched_factor_smem<float>(d, b, g.nm);
        if (sm > batched_max_smem()) return RCP_EUNSUPPORTED;
        g.grid = f64 ? batched_factor_grid<double>(d, b, g.nm, g.nt) : batched_factor_grid<float>(d, b, g.nm, g.nt);
        if (g.grid <= 0) return RCP_ECUDA;
        scr = std::max(scr, batched_factor_scratch_ints(b, g.nm) * (size_t)g.grid);
    }
    RCP_TRY(grow(h->bscr, scr * sizeof(int)));
    PhaseScope ps(h, s, PH_PANEL);
    for (int l = 0; l < nlegs; ++l) {
        const Leg &g = legs[l];
        if (f64)
            CU_TRY(launch_batched_factor<double>(batch, d, b, g.nm, n, A64, lda64, (double *const *)A, lda, Dd, Ds, perm,
                                                 (const double *)om, alpha, info, (const int *)h->bord.p,
                                                 (int *)h->bticket.p, (int *)h->bscr.p, g.grid, g.nt, g.first, g.last,
                                                 s));
        else
            CU_TRY(launch_batched_factor<float>(batch, d, b, g.nm, n, A64, lda64, (float *const *)A, lda, Dd, Ds, perm,
                                                (const float *)om, alpha, info, (const int *)h->bord.p,
                                                (int *)h->bticket.p, (int *)h->bscr.p, g.grid, g.nt, g.first, g.last,
                                                s));
    }
    return RCP_OK;
}

rcp_status rcp_set_batched_schedule(rcp_handle *h, int threads, int split) {
    if (!h || (threads != 0 && threads != 128 && threads != 256 && threads != 512) || split < 0 || split > 65535)
        return RCP_EINVAL;
    if (split > 0 && threads != 0 && threads != 512) return RCP_EINVAL;   // a split runs the large systems with 512 threads
    h->bt_nt = threads;
    h->bt_split = split;
    return RCP_OK;
}

rcp_status rcp_get_batched_schedule(rcp_handle *h, int nmax, int d, rcp_prec prec, int *b, int *d_out,
                                    int *threads, int *split) {
    if (!h || !valid_prec(prec)) return RCP_EINVAL;
    const int dkey = d > 0 ? d : 0, f64 = prec == RCP_FP64;
    int tb = 32, td = dkey > 0 ? dkey : std::min(32 + 8, 128), tn = 512, ts = 0;
    for (const auto &t : h->tuned)
        if (t.nmax == nmax && t.dkey == dkey && t.f64 == f64) { tb = t.b; td = t.d; tn = t.nt; ts = t.split; }
    if (h->bt_nt > 0 || h->bt_split > 0) {
        tn = h->bt_nt > 0 ? h->bt_nt : 512;
        ts = h->bt_split;
    }
    if (b) *b = tb;
    if (d_out) *d_out = td;
    if (threads) *threads = tn;
    if (split) *split = ts >= nmax ? 0 : ts;
    return RCP_OK;
}

rcp_status rcp_tune_batched(rcp_handle *h, int batch, int nmax, const int *n, const double *const *A64,
                            const int *lda64, void *const *A, const int *lda, double *const *Dd, double *const *Ds,
                            int *const *perm, const rcp_opts *opts, int *info, rcp_stream_t stream, int *best_b,
                            float *best_ms) {
    if (!h || !A64 || batch <= 0 || nmax <= 0) return RCP_EINVAL;
    const rcp_prec prec = opts ? opts->prec : RCP_FP64;
    if (!valid_prec(prec)) return RCP_EINVAL;
    const bool f64 = prec == RCP_FP64;
    const int dkey = (opts && opts->d > 0) ? opts->d : 0;   // 0: d = b + 8 follows each width
    cudaStream_t s = (cudaStream_t)stream;
    rcp_opts o = opts ? *opts : rcp_opts{};
    o.prec = prec;
    static const int cand[] = {8, 12, 16, 24, 32, 48, 64};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // schedules: {threads, split}: one launch of 512-thread CTAs; one of 256- or 128-thread CTAs
    // (tried where two, or three, fit an SM); the systems of order <= split in a second launch of
    // 256-thread CTAs
    const int sp = std::min(256, nmax / 2) & ~3;
    const int sched[4][2] = {{512, 0}, {256, 0}, {128, 0}, {512, sp}};
    const int keep_nt = h->bt_nt, keep_split = h->bt_split;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU_TRY(cudaEventCreate(&e0));
    CU_TRY(cudaEventCreate(&e1));
    int bb = 0, bd = 0, bnt = 512, bsp = 0;
    float bms = 0.f;
    rcp_status err = RCP_OK;
    for (int b : cand) {
        const int d = dkey > 0 ? dkey : std::min(b + 8, 128);
        const size_t smem = f64 ? batched_factor_smem<double>(d, b, nmax) : batched_factor_smem<float>(d, b, nmax);
        if (smem > batched_max_smem()) continue;
        for (const auto &sc : sched) {
            if (sc[0] < 512 && sc[1] == 0) {   // smaller CTAs only where more of them fit an SM
                const int g = f64 ? batched_factor_grid<double>(d, b, nmax, sc[0]) : batched_factor_grid<float>(d, b, nmax, sc[0]);
                if (g < (sc[0] == 256 ? 2 : 3) * sms) continue;
            }
            if (sc[1] > 0 && (sc[1] < 32 || sc[1] >= nmax)) continue;
            h->bt_nt = sc[0];
            h->bt_split = sc[1];
            o.b = b;
            o.d = d;
            err = rcp_factor_batched(h, batch, nmax, n, A64, lda64, A, lda, Dd, Ds, perm, &o, info, stream);   // warm-up
            if (err != RCP_OK) break;
            if (cudaEventRecord(e0, s) != cudaSuccess) { err = RCP_ECUDA; break; }
            err = rcp_factor_batched(h, batch, nmax, n, A64, lda64, A, lda, Dd, Ds, perm, &o, info, stream);
            if (err != RCP_OK) break;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { err = RCP_ECUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (bb == 0 || ms < bms) { bb = b; bd = d; bnt = sc[0]; bsp = sc[1]; bms = ms; }
        }
        if (err != RCP_OK) break;
    }
    h->bt_nt = keep_nt;
    h->bt_split = keep_split;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    if (err != RCP_OK) return err;
    if (bb == 0) return RCP_EUNSUPPORTED;
    bool found = false;
    for (auto &t : h->tuned)
        if (t.nmax == nmax && t.dkey == dkey && t.f64 == (int)f64) {
            t.b = bb; t.d = bd; t.nt = bnt; t.split = bsp; found = true;
        }
    if (!found) h->tuned.push_back({nmax, dkey, (int)f64, bb, bd, bnt, bsp});
    if (best_b) *best_b = bb;
    if (best_ms) *best_ms = bms;
    return RCP_OK;
}

rcp_status rcp_refine_batched(rcp_handle *h, int batch, int nmax, int nrhs, const int *n,
                              const double *const *A64, const int *lda64, const void *const *LA,
                              const int *ldla, const double *const *Dd, const double *const *Ds,
                              const int *const *perm, rcp_prec prec, const double *const *Bv, const int *ldb,
                              double *const *X, const int *ldx, double tol, int max_iter, double *berr,
                              int *iters, rcp_stream_t stream) {
    if (!h || batch < 0 || nmax < 0 || nmax > 65535 || nrhs < 0 || max_iter < 0 || !valid_prec(prec))
        return RCP_EINVAL;
    if (batch == 0 || nmax == 0 || nrhs == 0) return RCP_OK;
    if (!n || !LA || !ldla || !Dd || !Ds || !perm || !Bv || !ldb || !X || !ldx || (A64 && !lda64))
        return RCP_EINVAL;
    const bool f64 = prec == RCP_FP64;
    const size_t smem = f64 ? batched_refine_smem<double>(nrhs, nmax) : batched_refine_smem<float>(nrhs, nmax);
    if (smem > batched_max_smem()) return RCP_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    RCP_TRY(batched_order(h, batch, nmax, n, s));
    PhaseScope ps(h, s, A64 ? PH_RESIDUAL : PH_SOLVE);
    if (f64)
        CU_TRY(launch_batched_refine<double>(batch, nrhs, nmax, max_iter, tol, n, (const double *const *)LA, ldla, Dd,
                                             Ds, perm, A64, lda64, Bv, ldb, X, ldx, berr, iters,
                                             (const int *)h->bord.p, (int *)h->bticket.p, s));
    else
        CU_TRY(launch_batched_refine<float>(batch, nrhs, nmax, max_iter, tol, n, (const float *const *)LA, ldla, Dd,
                                            Ds, perm, A64, lda64, Bv, ldb, X, ldx, berr, iters,
                                            (const int *)h->bord.p, (int *)h->bticket.p, s));
    return RCP_OK;
}

rcp_status rcp_set_speculation(rcp_handle *h, int mode) {
    if (!h || mode < -1 || mode > 2) return RCP_EINVAL;
    h->spec_mode = mode;
    return RCP_OK;
}

rcp_status rcp_profile(rcp_handle *h, int enable) {
    if (!h) return RCP_EINVAL;
    h->profiling = enable < 0 ? 0 : (enable > 2 ? 2 : enable);
    return RCP_OK;
}

rcp_status rcp_profile_read(rcp_handle *h, double *ms, int *launches, int nphase) {
    if (!h || !ms || nphase < 1) return RCP_EINVAL;
    for (int i = 0; i < nphase; ++i) {
        ms[i] = 0.0;
        if (launches) launches[i] = 0;
    }
    for (auto &e : h->events) {
        CU_TRY(cudaEventSynchronize(e.b));
        float t = 0.f;
        CU_TRY(cudaEventElapsedTime(&t, e.a, e.b));
        if (e.phase < nphase) ms[e.phase] += t;
        h->pool.push_back(e.a);
        h->pool.push_back(e.b);
    }
    h->events.clear();
    for (int i = 0; i < nphase && i < PH_COUNT; ++i) {
        if (launches) launches[i] = h->launches[i];
        h->launches[i] = 0;
    }
    return RCP_OK;
}

rcp_status rcp_panel_trace(rcp_handle *h, unsigned long long *out, int cap) {
    if (!h || !out || cap < 0) return RCP_EINVAL;
    if (!h->trace.p) return RCP_EINVAL;
    size_t m = std::min((size_t)cap, (size_t)h->trace_n * PANEL_TRACE_SLOTS);
    CU_TRY(cudaDeviceSynchronize());
    CU_TRY(cudaMemcpy(out, h->trace.p, m * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return RCP_OK;
}

long long rcp_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

rcp_status rcp_l_norms(rcp_handle *h, int n, const void *LA, int lda, rcp_prec prec, rcp_stream_t stream,
                       double *norm1_L, double *norm1_Linv) {
    if (!h || n < 0 || !valid_prec(prec) || !norm1_L || !norm1_Linv || (n > 0 && (!LA || lda < n))) return RCP_EINVAL;
    *norm1_L = n > 0 ? 1.0 : 0.0;
    *norm1_Linv = *norm1_L;
    if (n == 0) return RCP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == RCP_FP64) return l_norms_impl<double>(h, n, (const double *)LA, lda, s, norm1_L, norm1_Linv);
    return l_norms_impl<float>(h, n, (const float *)LA, lda, s, norm1_L, norm1_Linv);
}

rcp_status rcp_exchange_latency(rcp_handle *h, int grid, int rounds, rcp_stream_t stream, double *us) {
    if (!h || !us || rounds < 1 || grid < 0) return RCP_EINVAL;
    *us = 0.0;
    const int maxg = exchange_probe_grid();
    if (grid == 0) grid = sm_count();
    if (maxg <= 0 || grid > maxg) return RCP_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    RCP_TRY(ensure_small(h));
    RCP_TRY(grow(h->keys, PANEL_KEY_WORDS * sizeof(unsigned long long)));
    unsigned *bar = (unsigned *)h->bar.p;
    unsigned long long *keys = (unsigned long long *)h->keys.p;
    int *status = (int *)h->status.p;
    auto reset = [&]() -> rcp_status {
        CU_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
        CU_TRY(cudaMemsetAsync(keys, 0, PANEL_KEY_WORDS * sizeof(unsigned long long), s));
        return RCP_OK;
    };
    CU_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    RCP_TRY(reset());
    CU_TRY(launch_exchange_probe(bar, keys, status, grid, std::min(rounds, 64), s));   // warm-up
    RCP_TRY(reset());
    cudaEvent_t e0, e1;
    CU_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return RCP_ECUDA;
    }
    cudaError_t ce = cudaEventRecord(e0, s);
    if (ce == cudaSuccess) ce = launch_exchange_probe(bar, keys, status, grid, rounds, s);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CU_TRY(ce);
    RCP_TRY(reset());
    int bits = 0;
    CU_TRY(cudaMemcpyAsync(&bits, status, sizeof bits, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    if (bits) return status_from_bits(bits);
    *us = 1e3 * (double)ms / rounds;
    return RCP_OK;
}

rcp_status rcp_wait_expiry(rcp_handle *h, int grid, int limit_us, rcp_stream_t stream, double *waited_us) {
    if (!h || !waited_us || grid < 0 || limit_us < 1 || limit_us > 2000000) return RCP_EINVAL;
    *waited_us = 0.0;
    const int maxg = exchange_probe_grid();
    if (grid == 0) grid = sm_count();
    if (maxg <= 0 || grid > maxg) return RCP_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    RCP_TRY(ensure_small(h));
    unsigned *bar = (unsigned *)h->bar.p;
    int *status = (int *)h->status.p;
    // the elapsed time goes to the refinement scalars' first word (not in use between calls)
    unsigned long long *el = (unsigned long long *)&((RefineScalars *)h->scal.p)->mx[0];
    CU_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    CU_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
    CU_TRY(cudaMemsetAsync(el, 0, sizeof *el, s));
    CU_TRY(launch_wait_expiry(bar, status, grid, (unsigned long long)limit_us * 1000ull, el, s));
    unsigned long long ns = 0;
    CU_TRY(cudaMemcpyAsync(&ns, el, sizeof ns, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    CU_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
    *waited_us = 1e-3 * (double)ns;
    return rcp_sync(h, stream);
}

rcp_status rcp_omega(int d, int n, uint64_t seed, double *omega, rcp_stream_t stream) {
    if (d < 1 || n < 0 || (n > 0 && !omega)) return RCP_EINVAL;
    CU_TRY(launch_omega<double>(d, n, seed, omega, (cudaStream_t)stream));
    return RCP_OK;
}

rcp_status rcp_sketch(int n, int d, const void *A, int lda, rcp_prec prec, uint64_t seed, const void *omega, void *B,
                      rcp_stream_t stream) {
    if (n < 0 || d < 1 || d > 128 || !valid_prec(prec) || (n > 0 && (!A || !B || lda < n))) return RCP_EINVAL;
    if (n == 0) return RCP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == RCP_FP64) {
        const double *om = (const double *)omega;
        double *tmp = nullptr;
        if (!om) {
            CU_TRY(cudaMallocAsync((void **)&tmp, (size_t)d * n * sizeof(double), s));
            CU_TRY(launch_omega<double>(d, n, seed, tmp, s));
            om = tmp;
        }
        cudaError_t e = launch_sketch<double, double>(n, d, (const double *)A, lda, om, (double *)B, nullptr, 0, s);
        if (tmp) cudaFreeAsync(tmp, s);
        CU_TRY(e);
    } else {
        const float *om = (const float *)omega;
        float *tmp = nullptr;
        if (!om) {
            CU_TRY(cudaMallocAsync((void **)&tmp, (size_t)d * n * sizeof(float), s));
            CU_TRY(launch_omega<float>(d, n, seed, tmp, s));
            om = tmp;
        }
        const bool tcs = tc_prec(prec);
        float *part = nullptr, *omt = nullptr;
        int *st = nullptr;
        const size_t pf = tcs ? sketch_tc_scratch_floats(n, d) : sketch_scratch_floats(n, d);
        bool ok = !(pf > 0 && cudaMallocAsync((void **)&part, pf * sizeof(float), s) != cudaSuccess);
        if (ok && tcs)
            ok = cudaMallocAsync((void **)&omt, sketch_tc_omega_floats(n, d) * sizeof(float), s) == cudaSuccess &&
                 cudaMallocAsync((void **)&st, sizeof(int), s) == cudaSuccess &&
                 cudaMemsetAsync(st, 0, sizeof(int), s) == cudaSuccess;
        cudaError_t e = cudaSuccess;
        if (ok && tcs) {
            e = launch_omega_split(n, d, om, omt, s);
            if (e == cudaSuccess)
                e = launch_sketch_tc(n, d, (const float *)A, lda, omt, (float *)B, part, part ? pf : 0, 0, n, st, s);
        } else if (ok) {
            e = launch_sketch<float, float>(n, d, (const float *)A, lda, om, (float *)B, part, part ? pf : 0, s);
        }
        if (!ok) cudaGetLastError();
        if (st) cudaFreeAsync(st, s);
        if (omt) cudaFreeAsync(omt, s);
        if (part) cudaFreeAsync(part, s);
        if (tmp) cudaFreeAsync(tmp, s);
        if (!ok) return RCP_ENOMEM;
        CU_TRY(e);
    }
    return RCP_OK;
}

}  // extern "C"
