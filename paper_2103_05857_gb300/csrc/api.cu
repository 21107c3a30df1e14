// api.cu -- the C ABI declared in include/sr_ot.h: handle, validation,
// workspace, and the host loop that drives the epoch and certificate kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/sr_ot.h"
#include "batched.h"
#include "common.cuh"
#include "internal.h"

using namespace srot;

namespace {

// Workspace slots owned by a handle; each grows on demand.
enum WsSlot {
    WS_Q = 0, WS_PARTIAL, WS_R64, WS_RQ32, WS_COLPART, WS_ROWPART, WS_CERT, WS_PERM, WS_PERMKEY,
    WS_PERMIDX, WS_GSTORE, WS_STATUS, WS_COST, WS_CHECK, WS_SCRATCH, WS_ATOMS, WS_B_INST,
    WS_B_QUEUE, WS_B_HEAD, WS_B_RES, WS_B_ATOMS, WS_B_BAD, WS_ADJ_INST, WS_ADJ_CP, WS_ADJ_RP, WS_TR_PART, WS_TR_ZERO, WS_TR_STATS, WS_FW_JS, WS_FW_UPART, WS_BF16, WS_BF16_ERR, WS_MET, WS_COST32, WS_FLOOR, WS_SB_STATE, WS_SB_Q, WS_SB_LIST, WS_COUNT
};

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

thread_local std::string g_create_error;

}  // namespace

namespace srot {
void set_handleless_error(const char *msg) { g_create_error = msg; }
}  // namespace srot

struct ProfPair {
    cudaEvent_t a, b;
    int kind;
};

struct sr_ot_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    DevBuf ws[WS_COUNT];
    double *h_cert = nullptr;   // pinned: kCertCount doubles
    int *h_status = nullptr;    // pinned: {device status, sparse-kernel resume index}
    double *h_check = nullptr;  // pinned: input check results
    long long launches = 0;     // kernels launched on this handle
    // profiling: event pairs waiting for the next synchronisation
    bool prof = false;
    std::vector<ProfPair> pending;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[SR_OT_PROF_KINDS] = {};
    long long prof_groups[SR_OT_PROF_KINDS] = {};
    // batched solves: side streams for concurrent tile launches, the tile
    // chosen per size bucket by the autotuner, captured graphs per shape set
    cudaStream_t side[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[4] = {nullptr, nullptr, nullptr, nullptr};
    std::map<long long, int> tuned_tile;
    std::map<unsigned long long, cudaGraphExec_t> graphs;
};

namespace {

sr_ot_status fail(sr_ot_handle h, sr_ot_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return st;
}

#define CK(h, expr)                                                                     \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail((h), e_ == cudaErrorMemoryAllocation ? SR_OT_ENOMEM : SR_OT_ECUDA, \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CKL(h)                                                                          \
    do {                                                                                \
        cudaError_t e_ = cudaPeekAtLastError();                                          \
        if (e_ != cudaSuccess) {                                                        \
            cudaGetLastError();                                                          \
            return fail((h), SR_OT_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                            \
        }                                                                               \
    } while (0)

cudaEvent_t prof_event(sr_ot_handle h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Bracket a launch group of class `kind` (no-op unless profiling).
struct ProfScope {
    sr_ot_handle h;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(sr_ot_handle h_, int kind_) : h(h_), kind(kind_) {
        if (h->prof) {
            a = prof_event(h);
            cudaEventRecord(a, h->stream);
        }
    }
    ~ProfScope() {
        if (h->prof) {
            cudaEvent_t b = prof_event(h);
            cudaEventRecord(b, h->stream);
            h->pending.push_back(ProfPair{a, b, kind});
        }
    }
};

// Fold finished event pairs into the totals (call after a stream sync).
void prof_collect(sr_ot_handle h) {
    for (auto &p : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            h->prof_ms[p.kind] += ms;
            h->prof_groups[p.kind] += 1;
        } else {
            cudaGetLastError();
        }
        h->event_pool.push_back(p.a);
        h->event_pool.push_back(p.b);
    }
    h->pending.clear();
}

sr_ot_status ws_get(sr_ot_handle h, int slot, size_t bytes, void **out) {
    DevBuf &b = h->ws[slot];
    bytes = std::max<size_t>(bytes, 256);
    if (b.cap < bytes) {
        if (b.p) {
            cudaStreamSynchronize(h->stream);
            cudaFree(b.p);
            b.p = nullptr;
            b.cap = 0;
        }
        size_t cap = bytes + bytes / 4;
        cudaError_t e = cudaMalloc(&b.p, cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, SR_OT_ENOMEM, "workspace allocation of %zu bytes failed: %s", cap,
                        cudaGetErrorString(e));
        }
        b.cap = cap;
    }
    *out = b.p;
    return SR_OT_OK;
}

template <typename T>
sr_ot_status ws_typed(sr_ot_handle h, int slot, size_t count, T **out) {
    void *p = nullptr;
    sr_ot_status st = ws_get(h, slot, count * sizeof(T), &p);
    *out = static_cast<T *>(p);
    return st;
}

// ---------------------------------------------------------------------------
// Input checks on the device: finiteness and sign of weights, finiteness of
// the cost source. out[0] = #bad entries of a, out[1] = #bad of b,
// out[2] = #non-finite cost entries.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_check_inputs(int m, int n, const Real *a, const Real *b, const Real *src,
                               long long nsrc, double *out) {
    __shared__ int cnt[3];
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
    __syncthreads();
    int c0 = 0, c1 = 0, c2 = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
         e < (long long)m || e < (long long)n || e < nsrc; e += (long long)gridDim.x * blockDim.x) {
        if (e < m) { Real v = a[e]; c0 += !(isfinite((double)v) && v >= Real(0)); }
        if (e < n) { Real v = b[e]; c1 += !(isfinite((double)v) && v >= Real(0)); }
        if (e < nsrc) c2 += !isfinite((double)src[e]);
    }
    if (c0) atomicAdd(&cnt[0], c0);
    if (c1) atomicAdd(&cnt[1], c1);
    if (c2) atomicAdd(&cnt[2], c2);
    __syncthreads();
    if (threadIdx.x < 3 && cnt[threadIdx.x]) atomicAdd(&out[threadIdx.x], (double)cnt[threadIdx.x]);
}

template <typename Real>
sr_ot_status check_inputs(sr_ot_handle h, int m, int n, const Real *a, const Real *b,
                          const Real *src, long long nsrc, const Real *src2, long long nsrc2) {
    double *d;
    sr_ot_status st = ws_typed(h, WS_CHECK, 4, &d);
    if (st) return st;
    CK(h, cudaMemsetAsync(d, 0, 4 * sizeof(double), h->stream));
    long long tot = std::max<long long>(std::max<long long>(m, n), nsrc);
    int blocks = (int)std::min<long long>((tot + 255) / 256, 152 * 8);
    k_check_inputs<Real><<<blocks, 256, 0, h->stream>>>(m, n, a, b, src, nsrc, d);
    h->launches += 1;
    CKL(h);
    if (src2 && nsrc2 > 0) {
        blocks = (int)std::min<long long>((nsrc2 + 255) / 256, 152 * 8);
        k_check_inputs<Real><<<blocks, 256, 0, h->stream>>>(0, 0, a, b, src2, nsrc2, d);
        h->launches += 1;
        CKL(h);
    }
    CK(h, cudaMemcpyAsync(h->h_check, d, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->h_check[0] > 0) return fail(h, SR_OT_EINVAL, "a has %.0f negative or non-finite entries", h->h_check[0]);
    if (h->h_check[1] > 0) return fail(h, SR_OT_EINVAL, "b has %.0f negative or non-finite entries", h->h_check[1]);
    if (h->h_check[2] > 0) return fail(h, SR_OT_ENUMERIC, "cost input has %.0f non-finite entries", h->h_check[2]);
    return SR_OT_OK;
}

sr_ot_status check_opts(sr_ot_handle h, const sr_ot_options *o) {
    if (!o) return fail(h, SR_OT_EINVAL, "opts is NULL");
    if (o->variant < SR_OT_BCFW || o->variant > SR_OT_FW) return fail(h, SR_OT_EINVAL, "unknown variant %d", o->variant);
    if (o->order < SR_OT_CYCLIC || o->order > SR_OT_GAP_ADAPTIVE) return fail(h, SR_OT_EINVAL, "unknown order %d", o->order);
    if (o->step != SR_OT_DEC && o->step != SR_OT_ELS) return fail(h, SR_OT_EINVAL, "unknown step rule %d", o->step);
    if (o->precision < SR_OT_FP64 || o->precision > SR_OT_FP32_BF16COST) return fail(h, SR_OT_EINVAL, "unknown precision %d", o->precision);
    if (!std::isfinite(o->rho) || o->rho < 0.0) return fail(h, SR_OT_EINVAL, "rho must be finite and >= 0 (got %g)", o->rho);
    if (!std::isfinite(o->tol_rel_gap) || o->tol_rel_gap < 0.0) return fail(h, SR_OT_EINVAL, "tol_rel_gap must be finite and >= 0");
    if (o->max_epochs < 0) return fail(h, SR_OT_EINVAL, "max_epochs must be >= 0");
    if (o->gap_every < 1) return fail(h, SR_OT_EINVAL, "gap_every must be >= 1");
    if (o->cert_schedule < 0 || o->cert_schedule > 1) return fail(h, SR_OT_EINVAL, "cert_schedule must be 0 or 1");
    if (o->refresh_every < 0) return fail(h, SR_OT_EINVAL, "refresh_every must be >= 0");
    if ((o->variant == SR_OT_BCAFW || o->variant == SR_OT_BCPFW) && o->step != SR_OT_ELS)
        return fail(h, SR_OT_EINVAL, "away and pairwise steps need the exact line search (SR_OT_ELS)");
    if (o->trace && o->trace_capacity < 0) return fail(h, SR_OT_EINVAL, "trace_capacity must be >= 0");
    if (o->epoch_kernel < SR_OT_EPOCH_AUTO || o->epoch_kernel > SR_OT_EPOCH_SPECULATIVE_SPLIT)
        return fail(h, SR_OT_EINVAL, "unknown epoch_kernel %d", o->epoch_kernel);
    if (o->cost_kind != SR_OT_COST_SQUARED && o->cost_kind != SR_OT_COST_EUCLIDEAN)
        return fail(h, SR_OT_EINVAL, "unknown cost_kind %d", o->cost_kind);
    if (o->spin_limit < 0) return fail(h, SR_OT_EINVAL, "spin_limit must be >= 0");
    return SR_OT_OK;
}

sr_ot_status check_stream_device(sr_ot_handle h) {
    int cur = -1;
    CK(h, cudaGetDevice(&cur));
    if (cur != h->device) CK(h, cudaSetDevice(h->device));
    return SR_OT_OK;
}

// Workspace and the certificate plan for an m x n instance.
sr_ot_status cert_work(sr_ot_handle h, int m, int n, CertWork *w) {
    int nchunks, rpc, ncolb, nrowb;
    cert_work_shape(m, n, &nchunks, &rpc, &ncolb, &nrowb);
    w->nchunks = nchunks;
    w->rows_per_chunk = rpc;
    w->ncolblocks = ncolb;
    w->nrowblocks = nrowb;
    sr_ot_status st;
    if ((st = ws_typed(h, WS_PARTIAL, (size_t)nchunks * n, &w->partial))) return st;
    if ((st = ws_typed(h, WS_R64, (size_t)n, &w->r64))) return st;
    if ((st = ws_typed(h, WS_RQ32, (size_t)n, &w->rq32))) return st;
    if ((st = ws_typed(h, WS_COLPART, (size_t)2 * ncolb, &w->colpart))) return st;
    if ((st = ws_typed(h, WS_ROWPART, (size_t)3 * nrowb, &w->rowpart))) return st;
    if ((st = ws_typed(h, WS_CERT, (size_t)kCertCount, &w->cert))) return st;
    return SR_OT_OK;
}

void fill_result(sr_ot_result *res, const double *cert, long long epochs, long long updates,
                 int status) {
    if (!res) return;
    res->objective = cert[kCertF];
    res->gap = cert[kCertG];
    res->rel_gap = cert[kCertRel];
    res->dual = cert[kCertW];
    res->row_err = cert[kCertFeas];
    res->epochs = epochs;
    res->block_updates = updates;
    res->status = status;
    res->reserved = 0;
}

// Resolve the cost source of an instance: C given, d = 3 points on the fly,
// or other d materialised once into the workspace.
template <typename Real>
sr_ot_status make_inst(sr_ot_handle h, const sr_ot_options *o, int m, int n, int d, const void *C,
                       const void *X, const void *Y, const void *a, const void *b, Inst<Real> *in) {
    in->m = m;
    in->n = n;
    in->a = static_cast<const Real *>(a);
    in->b = static_cast<const Real *>(b);
    in->C = nullptr;
    in->X = nullptr;
    in->Y = nullptr;
    const bool have_c = C != nullptr, have_pts = X != nullptr || Y != nullptr;
    if (have_c == have_pts) return fail(h, SR_OT_EINVAL, "pass exactly one of C or (X, Y)");
    sr_ot_status st;
    if (have_c) {
        if (o->precision == SR_OT_FP32_BF16COST)
            return fail(h, SR_OT_EINVAL, "SR_OT_FP32_BF16COST needs points X, Y, not C");
        in->cost_mode = kCostGiven;
        in->C = static_cast<const Real *>(C);
        if ((st = check_inputs<Real>(h, m, n, in->a, in->b, in->C, (long long)m * n, nullptr, 0))) return st;
        return SR_OT_OK;
    }
    if (!X || !Y) return fail(h, SR_OT_EINVAL, "points mode needs both X and Y");
    if (d <= 0) return fail(h, SR_OT_EINVAL, "d must be >= 1 in points mode (got %d)", d);
    const Real *Xr = static_cast<const Real *>(X), *Yr = static_cast<const Real *>(Y);
    if ((st = check_inputs<Real>(h, m, n, in->a, in->b, Xr, (long long)m * d, Yr, (long long)n * d))) return st;
    const bool euclid = o->cost_kind == SR_OT_COST_EUCLIDEAN;
    if (o->precision == SR_OT_FP32_BF16COST) {
        if (euclid) return fail(h, SR_OT_EUNSUPPORTED, "the BF16 cost is the squared one");
        if constexpr (std::is_same<Real, float>::value) {
            Real *Cw;
            if ((st = ws_typed(h, WS_COST, (size_t)m * n, &Cw))) return st;
            sr_ot_status s2 = sr_ot_cost_bf16(h, m, n, d, Xr, Yr, Cw);
            if (s2 != SR_OT_OK) return s2;
            in->cost_mode = kCostGiven;
            in->C = Cw;
            return SR_OT_OK;
        } else {
            return fail(h, SR_OT_EINVAL, "BF16 cost needs the FP32 element type");
        }
    }
    if (d == 3 && !euclid) {
        in->cost_mode = kCostPts3;
        in->X = Xr;
        in->Y = Yr;
        return SR_OT_OK;
    }
    Real *Cw;
    if ((st = ws_typed(h, WS_COST, (size_t)m * n, &Cw))) return st;
    {
        ProfScope ps(h, SR_OT_PROF_COST);
        launch_cost_plain<Real>(m, n, d, Xr, Yr, Cw, h->stream, euclid);
    }
    h->launches += 1;
    CKL(h);
    in->cost_mode = kCostGiven;
    in->C = Cw;
    return SR_OT_OK;
}

// Read back the certificate and the device status words (one sync).
// dev_status[0] is the status word, dev_status[1] the sparse-kernel resume index.
sr_ot_status read_cert(sr_ot_handle h, const CertWork &w, int *dev_status, int *dstat) {
    CK(h, cudaMemcpyAsync(h->h_cert, w.cert, kCertCount * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(h->h_status, dev_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *dstat = *h->h_status;
    prof_collect(h);
    return SR_OT_OK;
}

sr_ot_status dev_status_error(sr_ot_handle h, int dstat) {
    if (dstat == kDevNonFinite) return fail(h, SR_OT_ENUMERIC, "a non-finite gradient was met during the solve");
    if (dstat == kDevTimeout) return fail(h, SR_OT_ETIMEOUT, "a bounded device wait gave up");
    return fail(h, SR_OT_ECUDA, "device reported status %d", dstat);
}

// Full Frank-Wolfe (Alg. A.1): per iteration a certificate (which also gives
// every row's LMO vertex and the gap), then one global step.
template <typename Real>
sr_ot_status solve_fw_impl(sr_ot_handle h, const sr_ot_options *o, const Inst<Real> &in, Real *T,
                           int warm_start, sr_ot_result *res) {
    sr_ot_status st;
    const int m = in.m, n = in.n;
    double *q, *upart;
    int *js, *dstat_d;
    if ((st = ws_typed(h, WS_Q, (size_t)n, &q))) return st;
    if ((st = ws_typed(h, WS_STATUS, 4, &dstat_d))) return st;
    if ((st = ws_typed(h, WS_FW_JS, (size_t)m, &js))) return st;
    if ((st = ws_typed(h, WS_FW_UPART, (size_t)fw_upart_size(n) + 1, &upart))) return st;
    CK(h, cudaMemsetAsync(dstat_d, 0, sizeof(int), h->stream));
    CertWork w;
    if ((st = cert_work(h, m, n, &w))) return st;
    launch_init_plan<Real>(in, T, warm_start, o->rho, q, h->stream);
    h->launches += warm_start ? 1 : 2;
    CKL(h);
    double *gamma_dev = upart + fw_upart_size(n);
    long long it = 0;
    bool converged = false;
    for (it = 0; it < o->max_epochs; ++it) {
        {
            ProfScope ps(h, SR_OT_PROF_CERT);
            launch_certificate<Real>(in, T, o->rho, o->tol_rel_gap, w, nullptr, nullptr, h->stream, js);
        }
        h->launches += 4;
        CKL(h);
        int dstat = 0;
        if ((st = read_cert(h, w, dstat_d, &dstat))) return st;
        if (!std::isfinite(h->h_cert[kCertG])) return fail(h, SR_OT_ENUMERIC, "non-finite gap at iteration %lld", it);
        if (h->h_cert[kCertStop] != 0.0) { converged = true; break; }
        {
            ProfScope ps(h, SR_OT_PROF_EPOCH);
            launch_fw_step<Real>(in, T, js, w.r64, w.cert, o->step, it, o->rho, upart, gamma_dev, h->stream);
        }
        h->launches += o->step == SR_OT_ELS ? 3 : 2;
        CKL(h);
    }
    if (!converged) {
        launch_certificate<Real>(in, T, o->rho, o->tol_rel_gap, w, nullptr, nullptr, h->stream);
        h->launches += 4;
        CKL(h);
        int dstat = 0;
        if ((st = read_cert(h, w, dstat_d, &dstat))) return st;
        converged = h->h_cert[kCertStop] != 0.0;
    }
    sr_ot_status out = (o->tol_rel_gap > 0.0 && !converged) ? SR_OT_NOT_CONVERGED : SR_OT_OK;
    fill_result(res, h->h_cert, it, it * (long long)m, out);
    return out;
}

template <typename Real>
sr_ot_status solve_impl(sr_ot_handle h, const sr_ot_options *o, int m, int n, int d, const void *C,
                        const void *X, const void *Y, const void *a, const void *b, void *T_inout,
                        int warm_start, sr_ot_result *res) {
    sr_ot_status st;
    Inst<Real> in;
    if ((st = make_inst<Real>(h, o, m, n, d, C, X, Y, a, b, &in))) return st;
    const bool fp64 = std::is_same<Real, double>::value;
    if (o->variant == SR_OT_FW) return solve_fw_impl<Real>(h, o, in, static_cast<Real *>(T_inout), warm_start, res);
    const bool ga = o->order == SR_OT_GAP_ADAPTIVE;
    if (ga && m > epoch_ga_max_m())
        return fail(h, SR_OT_EUNSUPPORTED, "gap-adaptive sampling takes m <= %d (got %d)", epoch_ga_max_m(), m);
    if (n > epoch_max_n(fp64))
        return fail(h, SR_OT_EUNSUPPORTED, "n = %d exceeds the single-instance limit %d for this precision",
                    n, epoch_max_n(fp64));
    // FP64 BCFW on rows of width <= 512 runs on the single-warp kernel, which
    // streams the cost row: d = 3 points are turned into C once (the same
    // FP64 operations in the same order as the point cost, so the values are
    // identical) and the whole solve, certificate included, reads C.
    bool f64w = false;
    float *c32 = nullptr;
    if constexpr (std::is_same<Real, double>::value) {
        if (o->variant == SR_OT_BCFW && !ga && n <= epoch_f64w_max_n() &&
            (size_t)m * n * (sizeof(double) + sizeof(float)) <= ((size_t)1 << 30)) {
            if (in.cost_mode == kCostPts3) {
                double *Cw;
                if ((st = ws_typed(h, WS_COST, (size_t)m * n, &Cw))) return st;
                {
                    ProfScope ps(h, SR_OT_PROF_COST);
                    launch_cost_plain<double>(m, n, 3, in.X, in.Y, Cw, h->stream, false);
                }
                h->launches += 1;
                CKL(h);
                in.C = Cw;
                in.cost_mode = kCostGiven;
            }
            if (in.cost_mode == kCostGiven) {
                // its FP32 rounding, for the kernel's argmin screen
                if ((st = ws_typed(h, WS_COST32, (size_t)m * n, &c32))) return st;
                launch_round_cost(in.C, c32, (size_t)m * n, h->stream);
                h->launches += 1;
                CKL(h);
                f64w = true;
            }
        }
    }
    Real *T = static_cast<Real *>(T_inout);
    double *q;
    int *dstat_d;
    if ((st = ws_typed(h, WS_Q, (size_t)n, &q))) return st;
    if ((st = ws_typed(h, WS_STATUS, 4, &dstat_d))) return st;
    CK(h, cudaMemsetAsync(dstat_d, 0, sizeof(int), h->stream));
    CK(h, cudaMemsetAsync(dstat_d + 1, 0xff, sizeof(int), h->stream));  // resume = -1
    CK(h, cudaMemsetAsync(dstat_d + 3, 0, sizeof(int), h->stream));     // no record overflow yet
    CertWork w;
    if ((st = cert_work(h, m, n, &w))) return st;
    int *perm = nullptr;
    uint64_t *pkey = nullptr;
    int *pidx = nullptr;
    if (o->order == SR_OT_PERMUTE) {
        if ((st = ws_typed(h, WS_PERM, (size_t)m, &perm))) return st;
        size_t sb = make_perm_scratch_bytes(m);
        if (sb) {
            int L = 1;
            while (L < m) L <<= 1;
            if ((st = ws_typed(h, WS_PERMKEY, (size_t)L, &pkey))) return st;
            if ((st = ws_typed(h, WS_PERMIDX, (size_t)L, &pidx))) return st;
        }
    }
    launch_init_plan<Real>(in, T, warm_start, o->rho, q, h->stream);
    h->launches += warm_start ? 1 : 2;
    CKL(h);

    // Away / pairwise steps in FP32 run on the active-set kernel while every
    // row fits its atom record; an overflow hands the rest of the solve to
    // the dense kernel.
    bool use_sparse = false;
    int4 *atoms = nullptr;
    if constexpr (std::is_same<Real, float>::value) {
        if ((o->variant == SR_OT_BCAFW || o->variant == SR_OT_BCPFW) && !o->dense_only && !ga &&
            n <= epoch_max_n(false)) {
            if ((st = ws_typed(h, WS_ATOMS, (size_t)m * kAtomRecord, &atoms))) return st;
            CK(h, cudaMemsetAsync(dstat_d + 2, 0, sizeof(int), h->stream));
            launch_build_atoms(m, n, T, atoms, dstat_d + 2, h->stream);
            h->launches += 1;
            CKL(h);
            int ovf = 0;
            CK(h, cudaMemcpyAsync(h->h_status, dstat_d + 2, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            ovf = h->h_status[0];
            use_sparse = (ovf == 0);
        }
    }

    EpochArgs<Real> A;
    A.in = in;
    A.T = T;
    A.q = q;
    A.rho = o->rho;
    A.variant = o->variant;
    A.step = o->step;
    A.order = o->order;
    A.seed = o->seed;
    A.perm = perm;
    A.g_store = nullptr;
    A.ga_inner = 0;
    const int ga_every = o->ga_global_only ? 1 : std::max(1, o->ga_M);
    if (ga) {
        // every g_i exact at the start (the reading of Alg. A.4's initialisation)
        if ((st = ws_typed(h, WS_GSTORE, (size_t)m, &A.g_store))) return st;
        A.ga_inner = o->ga_global_only ? 0 : 1;
        launch_certificate<Real>(in, T, o->rho, o->tol_rel_gap, w, nullptr, A.g_store, h->stream);
        h->launches += 4;
        CKL(h);
    }
    A.trace = o->trace;
    A.trace_cap = o->trace ? o->trace_capacity : 0;
    A.status = dstat_d;
    A.atoms = atoms;
    A.resume = nullptr;
    A.resume_in = nullptr;
    A.sticky = dstat_d + 3;
    A.spin_limit = o->spin_limit;
    A.gate = o->start_gate;
    A.C32 = c32;
    {
        const size_t rb = (size_t)n * sizeof(Real);
        bool v = (rb % 16 == 0) && ((uintptr_t)T % 16 == 0);
        if (in.cost_mode == kCostGiven) v = v && ((uintptr_t)in.C % 16 == 0);
        A.vec = v;
    }

    const int refresh_every = fp64 ? 0 : o->refresh_every;
    // cert_schedule 1: the next certificate when the gap's geometric decay
    // since the last one predicts the tolerance (at least 1, at most 8
    // certificate periods on); an overflow of the active sets needs no
    // certificate any more (the kernels switch to the dense one themselves)
    const bool predicted = o->cert_schedule == 1 && o->tol_rel_gap > 0.0 && !ga;
    long long next_cert = 0, ep_prev = 0;
    double g_prev = 0.0;
    long long ep = 0, ncert = 0;
    bool converged = false, have_cert = false;
    for (ep = 0; ep < o->max_epochs; ++ep) {
        if (o->order == SR_OT_PERMUTE) {
            launch_make_perm(o->seed, ep, m, perm, pkey, pidx, h->stream);
            h->launches += make_perm_scratch_bytes(m) ? 2 : 1;
            CKL(h);
        }
        A.k0 = ep * (long long)m;
        A.epoch = ep;
        {
            ProfScope ps(h, SR_OT_PROF_EPOCH);
            if (ga) {
                launch_epoch_ga<Real>(A, h->stream);
            } else if constexpr (std::is_same<Real, float>::value) {
                if (use_sparse) {
                    EpochArgs<float> As = A;
                    As.resume = dstat_d + 1;
                    const int ek = o->epoch_kernel;
                    bool ran = false;
                    if (ek == SR_OT_EPOCH_AUTO)  // uniform order: only the split chain takes it
                        ran = launch_epoch_spec(As, h->stream, o->order == SR_OT_UNIFORM ? kSpecChainSplit : 3);
                    else if (ek == SR_OT_EPOCH_SPECULATIVE)
                        ran = launch_epoch_spec(As, h->stream, 3);
                    else if (ek == SR_OT_EPOCH_SPECULATIVE_ONE_CHAIN)
                        ran = launch_epoch_spec(As, h->stream, 1);
                    else if (ek == SR_OT_EPOCH_SPECULATIVE_SPLIT)
                        ran = launch_epoch_spec(As, h->stream, kSpecChainSplit);
                    if (!ran && ek != SR_OT_EPOCH_TWO_PHASE) ran = launch_epoch_pipe(As, h->stream);
                    if (!ran) launch_epoch_sparse(As, h->stream);
                    EpochArgs<float> Ad = A;
                    Ad.resume_in = dstat_d + 1;  // finishes the epoch only after an overflow
                    launch_epoch<float>(Ad, h->stream);
                    h->launches += 1;
                } else {
                    launch_epoch<Real>(A, h->stream);
                }
            } else if constexpr (std::is_same<Real, double>::value) {
                if (!(f64w && launch_epoch_f64w(A, h->stream))) launch_epoch<Real>(A, h->stream);
            } else {
                launch_epoch<Real>(A, h->stream);
            }
        }
        h->launches += 1;
        CKL(h);
        const bool last = ep + 1 == o->max_epochs;
        const bool ga_global = ga && (ep + 1) % ga_every == 0;  // every g_i again (Alg. A.4)
        const bool cert_due = predicted ? ((ep + 1) % o->gap_every == 0 && ep + 1 >= next_cert) || last
                                        : (ep + 1) % o->gap_every == 0 || last;
        if (ga_global && !cert_due) {
            ProfScope ps(h, SR_OT_PROF_CERT);
            launch_certificate<Real>(in, T, o->rho, o->tol_rel_gap, w, nullptr, A.g_store, h->stream);
            h->launches += 4;
            CKL(h);
        }
        if (cert_due) {
            ++ncert;
            double *refresh = (refresh_every > 0 && ncert % refresh_every == 0) ? q : nullptr;
            {
                ProfScope ps(h, SR_OT_PROF_CERT);
                launch_certificate<Real>(in, T, o->rho, o->tol_rel_gap, w, refresh,
                                         ga_global ? A.g_store : nullptr, h->stream);
            }
            h->launches += 4;
            CKL(h);
            // Without a tolerance nothing on the host depends on an
            // intermediate certificate (an active-set solve still reads each
            // one for a row that outgrew its record): the stream runs on and
            // only the last one is read back.
            if (!last && o->tol_rel_gap == 0.0 && !use_sparse) continue;
            int dstat = 0;
            if ((st = read_cert(h, w, dstat_d, &dstat))) return st;
            have_cert = true;
            if (dstat) return dev_status_error(h, dstat);
            if (use_sparse && h->h_status[1] >= 0) use_sparse = false;  // a row outgrew its record
            if (h->h_cert[kCertStop] != 0.0) { converged = true; ++ep; break; }
            if (predicted) {
                const double f = h->h_cert[kCertF], g = h->h_cert[kCertG];
                long long skip = 1;
                if (g_prev > 0.0 && g > 0.0 && g < g_prev && ep + 1 > ep_prev && f > 0.0) {
                    const double rate = std::log(g / g_prev) / (double)(ep + 1 - ep_prev);  // < 0
                    const double early = 0.75 * std::log(o->tol_rel_gap * f / g) / rate;   // epochs, > 0
                    skip = early >= 8.0 * o->gap_every ? 8 * (long long)o->gap_every
                                                         : (early < 1.0 ? 1 : (long long)early);
                }
                g_prev = g;
                ep_prev = ep + 1;
                next_cert = ep + 1 + skip;
            }
        }
    }
    if (!have_cert) {
        launch_certificate<Real>(in, T, o->rho, o->tol_rel_gap, w, nullptr, nullptr, h->stream);
        h->launches += 4;
        CKL(h);
        int dstat = 0;
        if ((st = read_cert(h, w, dstat_d, &dstat))) return st;
        if (dstat) return dev_status_error(h, dstat);
        converged = h->h_cert[kCertStop] != 0.0;
    }
    sr_ot_status out = (o->tol_rel_gap > 0.0 && !converged) ? SR_OT_NOT_CONVERGED : SR_OT_OK;
    fill_result(res, h->h_cert, ep, ep * (long long)m, out);
    return out;
}

template <typename Real>
sr_ot_status gap_impl(sr_ot_handle h, const sr_ot_options *o, int m, int n, int d, const void *C,
                      const void *X, const void *Y, const void *a, const void *b, const void *T,
                      double *g_rows, sr_ot_result *res) {
    sr_ot_status st;
    Inst<Real> in;
    if ((st = make_inst<Real>(h, o, m, n, d, C, X, Y, a, b, &in))) return st;
    CertWork w;
    if ((st = cert_work(h, m, n, &w))) return st;
    int *dstat_d;
    if ((st = ws_typed(h, WS_STATUS, 1, &dstat_d))) return st;
    CK(h, cudaMemsetAsync(dstat_d, 0, sizeof(int), h->stream));
    {
        ProfScope ps(h, SR_OT_PROF_CERT);
        launch_certificate<Real>(in, static_cast<const Real *>(T), o->rho, o->tol_rel_gap, w, nullptr,
                                 g_rows, h->stream);
    }
    h->launches += 4;
    CKL(h);
    int dstat = 0;
    if ((st = read_cert(h, w, dstat_d, &dstat))) return st;
    fill_result(res, h->h_cert, 0, 0, SR_OT_OK);
    return SR_OT_OK;
}

sr_ot_status check_sizes(sr_ot_handle h, int m, int n) {
    if (m <= 0 || n <= 0) return fail(h, SR_OT_EINVAL, "m and n must be >= 1 (got m=%d, n=%d)", m, n);
    return SR_OT_OK;
}


// ---------------------------------------------------------------------------
// Batched solve
// ---------------------------------------------------------------------------
// Size buckets by n and the tile shapes the autotuner tries for each.
constexpr int kNumBuckets = 4;
const int kBucketMaxN[kNumBuckets] = {256, 512, 1024, 2048};
const std::vector<int> kBucketTiles[kNumBuckets] = {{0, 1, 2}, {1, 2, 3}, {3, 4}, {5, 6}};

int bucket_of(int n) {
    for (int k = 0; k < kNumBuckets; ++k)
        if (n <= kBucketMaxN[k]) return k;
    return -1;
}

__global__ void k_batch_check(const BatchInst *inst, int batch, const float *X, const float *Y,
                              const float *a, const float *b, int *bad) {
    for (int k = blockIdx.x; k < batch; k += gridDim.x) {
        const BatchInst I = inst[k];
        int c = 0;
        for (int e = threadIdx.x; e < I.m; e += blockDim.x) {
            const float v = a[I.off_a + e];
            c += !(isfinite(v) && v >= 0.f);
            for (int t = 0; t < 3; ++t) c += !isfinite(X[I.off_X + 3 * (long long)e + t]);
        }
        for (int e = threadIdx.x; e < I.n; e += blockDim.x) {
            const float v = b[I.off_b + e];
            c += !(isfinite(v) && v >= 0.f);
            for (int t = 0; t < 3; ++t) c += !isfinite(Y[I.off_Y + 3 * (long long)e + t]);
        }
        if (c) atomicAdd(&bad[k], c);
    }
}

// ---------------------------------------------------------------------------
// Envelope-theorem gradients (adjoint pass) for one or many instances.
// ---------------------------------------------------------------------------
template <typename Real>
sr_ot_status adjoint_impl(sr_ot_handle h, const sr_ot_options *o, int ninst, const int *m, const int *n,
                          int d, const long long *oX, const long long *oY, const long long *ob,
                          const long long *oT, const long long *oa, const void *X, const void *Y,
                          const void *a, const void *b, const void *T, void *dC, void *dX, void *dY, void *db,
                          void *xhat, double *stats) {
    if (!o) return fail(h, SR_OT_EINVAL, "opts is NULL");
    if (!std::isfinite(o->rho) || o->rho < 0.0) return fail(h, SR_OT_EINVAL, "rho must be finite and >= 0");
    if (!T) return fail(h, SR_OT_EINVAL, "T must be non-NULL");
    if ((dX || dY) && (!X || !Y)) return fail(h, SR_OT_EINVAL, "dX and dY need the points X and Y");
    if (db && !b) return fail(h, SR_OT_EINVAL, "db needs b");
    if (xhat && !Y) return fail(h, SR_OT_EINVAL, "the barycentric projection needs the points Y");
    if (stats && (!a || !b)) return fail(h, SR_OT_EINVAL, "the transfer statistics need a and b");
    if ((dX || dY) && o->cost_kind != SR_OT_COST_SQUARED)
        return fail(h, SR_OT_EUNSUPPORTED, "the point gradients dX, dY are those of the squared cost");
    if ((dX || dY || xhat) && (d < 1 || d > 31)) return fail(h, SR_OT_EUNSUPPORTED, "point outputs take 1 <= d <= 31 (got %d)", d);
    if (!(dX || dY || xhat) && (d < 1 || d > 31)) d = 3;  // d unused: no point outputs requested
    if (!dC && !dX && !dY && !db && !xhat && !stats) return SR_OT_OK;
    for (int k = 0; k < ninst; ++k) {
        if (m[k] <= 0 || n[k] <= 0) return fail(h, SR_OT_EINVAL, "instance %d: m and n must be >= 1", k);
        if (oX[k] < 0 || oY[k] < 0 || ob[k] < 0 || oT[k] < 0 || oa[k] < 0) return fail(h, SR_OT_EINVAL, "instance %d: negative offset", k);
    }
    std::vector<AdjInst> inst(ninst);
    const AdjTotals tot = adj_plan(ninst, m, n, d, (int)sizeof(Real), inst.data());
    if (tot.tiles > 0x7FFFFFFFLL) return fail(h, SR_OT_EUNSUPPORTED, "adjoint launch too large (%lld tiles)", tot.tiles);
    for (int k = 0; k < ninst; ++k) {
        inst[k].oX = oX[k];
        inst[k].oY = oY[k];
        inst[k].ob = ob[k];
        inst[k].oT = oT[k];
        inst[k].oa = oa[k];
    }
    sr_ot_status st;
    AdjInst *d_inst;
    Real *cp, *rp;
    if ((st = ws_typed(h, WS_ADJ_INST, (size_t)ninst, &d_inst))) return st;
    if ((st = ws_typed(h, WS_ADJ_CP, (size_t)tot.colpart, &cp))) return st;
    if ((st = ws_typed(h, WS_ADJ_RP, (size_t)tot.rowpart, &rp))) return st;
    CK(h, cudaMemcpyAsync(d_inst, inst.data(), sizeof(AdjInst) * ninst, cudaMemcpyHostToDevice, h->stream));
    double *tpart = nullptr, *tstats = nullptr;
    unsigned long long *zeros = nullptr;
    if (stats) {
        if ((st = ws_typed(h, WS_TR_PART, (size_t)tot.fin_blocks, &tpart))) return st;
        if ((st = ws_typed(h, WS_TR_ZERO, (size_t)ninst, &zeros))) return st;
        if ((st = ws_typed(h, WS_TR_STATS, (size_t)4 * ninst, &tstats))) return st;
        CK(h, cudaMemsetAsync(zeros, 0, sizeof(unsigned long long) * ninst, h->stream));
    }
    AdjArgs<Real> A;
    A.inst = d_inst;
    A.ninst = ninst;
    A.d = d;
    A.rho = o->rho;
    A.X = static_cast<const Real *>(X);
    A.Y = static_cast<const Real *>(Y);
    A.b = static_cast<const Real *>(b);
    A.T = static_cast<const Real *>(T);
    A.dC = static_cast<Real *>(dC);
    A.dX = static_cast<Real *>(dX);
    A.dY = static_cast<Real *>(dY);
    A.db = static_cast<Real *>(db);
    A.colpart = cp;
    A.rowpart = rp;
    A.xhat = static_cast<Real *>(xhat);
    A.a = static_cast<const Real *>(a);
    A.tpart = tpart;
    A.zeros = zeros;
    A.tstats = tstats;
    A.total_tiles = (int)tot.tiles;
    A.total_cols = tot.cols;
    A.total_rows = tot.rows;
    A.total_fin = (int)tot.fin_blocks;
    {
        ProfScope ps(h, SR_OT_PROF_GRAD);
        if (!launch_adjoint<Real>(A, h->stream)) return fail(h, SR_OT_EUNSUPPORTED, "d = %d out of range", d);
    }
    h->launches += 1 + ((dX || dY || db || xhat || stats) ? 1 : 0) + (stats ? 1 : 0);
    CKL(h);
    if (stats) CK(h, cudaMemcpyAsync(stats, tstats, sizeof(double) * 4 * ninst, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return SR_OT_OK;
}

template <typename Real>
sr_ot_status grad_impl(sr_ot_handle h, const sr_ot_options *o, int ninst, const int *m, const int *n,
                       int d, const long long *oX, const long long *oY, const long long *ob,
                       const long long *oT, const void *X, const void *Y, const void *b, const void *T,
                       void *dC, void *dX, void *dY, void *db) {
    std::vector<long long> oa(ninst > 0 ? ninst : 1, 0);
    return adjoint_impl<Real>(h, o, ninst, m, n, d, oX, oY, ob, oT, oa.data(), X, Y, nullptr, b, T, dC, dX, dY,
                              db, nullptr, nullptr);
}

sr_ot_status ensure_side_streams(sr_ot_handle h) {
    if (h->ev_fork) return SR_OT_OK;
    for (int k = 0; k < 4; ++k) {
        CK(h, cudaStreamCreateWithFlags(&h->side[k], cudaStreamNonBlocking));
        CK(h, cudaEventCreateWithFlags(&h->ev_join[k], cudaEventDisableTiming));
    }
    CK(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    return SR_OT_OK;
}

// The batched speculative form (see solve_spec_batch.cu): instances with
// n <= 4096 in width buckets; one set-up launch, then one launch per bucket
// (each on its own side stream) in which every CTA solves one instance to
// its stopping rule. Instances it does not take (n above the widths, or a
// row that outgrew its record) are appended to `solo`.
sr_ot_status solve_batched_spec(sr_ot_handle h, const sr_ot_options *o, int batch, const int *m, const int *n,
                                const std::vector<BatchInst> &inst, const BatchInst *d_inst, int4 *d_atoms,
                                const float *X, const float *Y, const float *a, const float *b, float *T,
                                sr_ot_result *res, std::vector<int> &solo) {
    sr_ot_status st;
    std::vector<std::vector<int>> bq(kSpecBatchBuckets);
    long long qlen = 1;
    for (int k = 0; k < batch; ++k) {
        const int bk = spec_batch_bucket(n[k]);
        if (bk < 0) { solo.push_back(k); continue; }
        bq[bk].push_back(k);
        qlen = std::max(qlen, inst[k].off_b + n[k]);
    }
    // longest epoch first within a bucket (the hardware starts CTAs in index
    // order): an update costs about the same at every width of a bucket, so
    // an instance's chain is m updates per epoch
    auto by_chain = [&](int x, int y) { return m[x] != m[y] ? m[x] > m[y] : n[x] > n[y]; };
    for (auto &v : bq) std::stable_sort(v.begin(), v.end(), by_chain);
    std::vector<int> hlist, lstart(kSpecBatchBuckets + 1, 0);
    for (int bk = 0; bk < kSpecBatchBuckets; ++bk) {
        lstart[bk] = (int)hlist.size();
        hlist.insert(hlist.end(), bq[bk].begin(), bq[bk].end());
    }
    lstart[kSpecBatchBuckets] = (int)hlist.size();
    if (hlist.empty()) return SR_OT_OK;
    SpecInstState *d_state;
    double *d_q;
    int *d_list;
    if ((st = ws_typed(h, WS_SB_STATE, (size_t)batch, &d_state))) return st;
    if ((st = ws_typed(h, WS_SB_Q, (size_t)qlen, &d_q))) return st;
    if ((st = ws_typed(h, WS_SB_LIST, (size_t)batch, &d_list))) return st;
    CK(h, cudaMemcpyAsync(d_list, hlist.data(), sizeof(int) * hlist.size(), cudaMemcpyHostToDevice, h->stream));
    SpecBatchArgs B{};
    B.inst = d_inst;
    B.list = d_list;
    B.state = d_state;
    B.q = d_q;
    B.X = X;
    B.Y = Y;
    B.a = a;
    B.b = b;
    B.T = T;
    B.atoms = d_atoms;
    B.rho = o->rho;
    B.tol = o->tol_rel_gap;
    B.max_epochs = o->max_epochs;
    B.gap_every = o->gap_every;
    B.warm = o->batch_warm_start ? 1 : 0;
    const bool uniform = o->order == SR_OT_UNIFORM;
    {
        ProfScope ps(h, SR_OT_PROF_BATCH);
        launch_spec_batch_init(B, (int)hlist.size(), h->stream);
        h->launches += 1;
        CKL(h);
        CK(h, cudaEventRecord(h->ev_fork, h->stream));
        int used = 0;
        // widest bucket first: its CTAs are dispatched first and its (larger)
        // instances start at once
        for (int bk = kSpecBatchBuckets - 1; bk >= 0; --bk) {
            const int cnt = lstart[bk + 1] - lstart[bk];
            if (cnt == 0) continue;
            cudaStream_t s = h->side[used];
            CK(h, cudaStreamWaitEvent(s, h->ev_fork, 0));
            SpecBatchArgs Bb = B;
            Bb.list = d_list + lstart[bk];
            if (!launch_spec_batch_solve(bk, uniform, Bb, cnt, o->seed, o->spin_limit, s))
                return fail(h, SR_OT_EUNSUPPORTED, "no speculative kernel for width bucket %d", bk);
            h->launches += 1;
            CKL(h);
            CK(h, cudaEventRecord(h->ev_join[used], s));
            CK(h, cudaStreamWaitEvent(h->stream, h->ev_join[used], 0));
            ++used;
        }
    }
    std::vector<SpecInstState> hs(batch);
    CK(h, cudaMemcpyAsync(hs.data(), d_state, sizeof(SpecInstState) * batch, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    prof_collect(h);
    for (int k = 0; k < batch; ++k) {
        if (spec_batch_bucket(n[k]) < 0) continue;
        const SpecInstState &r = hs[k];
        if (r.active) return fail(h, SR_OT_ECUDA, "instance %d still running after its solve", k);
        sr_ot_result &o2 = res[k];
        o2.objective = r.f;
        o2.gap = r.g;
        o2.rel_gap = r.f != 0.0 ? r.g / r.f : 0.0;
        o2.dual = r.f - r.g;
        o2.row_err = r.feas;
        o2.epochs = r.ep;
        o2.block_updates = r.updates;
        o2.reserved = 0;
        o2.status = r.status == kInstOk ? SR_OT_OK
                  : r.status == kInstNotConverged ? SR_OT_NOT_CONVERGED
                  : r.status == kInstNonFinite ? SR_OT_ENUMERIC
                  : r.status == kInstTimeout ? SR_OT_ETIMEOUT : SR_OT_OK;
        if (r.status == kInstNeedsDense) solo.push_back(k);
    }
    return SR_OT_OK;
}

sr_ot_status solve_batched_impl(sr_ot_handle h, const sr_ot_options *o, int batch, const int *m,
                                const int *n, int d, const long long *off_X, const long long *off_Y,
                                const long long *off_a, const long long *off_b,
                                const long long *off_T, const float *X, const float *Y,
                                const float *a, const float *b, float *T, sr_ot_result *res) {
    if (batch <= 0) return fail(h, SR_OT_EINVAL, "batch must be >= 1");
    if (!m || !n || !off_X || !off_Y || !off_a || !off_b || !off_T || !res)
        return fail(h, SR_OT_EINVAL, "size, offset and result arrays must be non-NULL");
    if (!X || !Y || !a || !b || !T) return fail(h, SR_OT_EINVAL, "X, Y, a, b, T must be non-NULL");
    if (d != 3) return fail(h, SR_OT_EUNSUPPORTED, "batched solves take points with d = 3 (got %d)", d);
    if (o->precision != SR_OT_FP32) return fail(h, SR_OT_EUNSUPPORTED, "batched solves run in SR_OT_FP32");
    if (o->cost_kind != SR_OT_COST_SQUARED) return fail(h, SR_OT_EUNSUPPORTED, "batched solves take the squared cost");
    if (o->variant == SR_OT_FW) return fail(h, SR_OT_EUNSUPPORTED, "batched solves run the block-coordinate variants");
    if (o->order == SR_OT_GAP_ADAPTIVE) return fail(h, SR_OT_EUNSUPPORTED, "batched solves take cyclic, permuted or uniform order");
    sr_ot_status st;
    // ---- descriptors, size checks, buckets --------------------------------
    std::vector<BatchInst> inst(batch);
    std::vector<std::vector<int>> buckets(kNumBuckets);
    std::vector<int> solo;  // instances solved one at a time (n above the tile widths)
    long long atoms_total = 0;
    for (int k = 0; k < batch; ++k) {
        if (m[k] <= 0 || n[k] <= 0) return fail(h, SR_OT_EINVAL, "instance %d: m and n must be >= 1", k);
        if (off_X[k] < 0 || off_Y[k] < 0 || off_a[k] < 0 || off_b[k] < 0 || off_T[k] < 0)
            return fail(h, SR_OT_EINVAL, "instance %d: negative offset", k);
        if (o->order == SR_OT_PERMUTE && m[k] > 2048)
            return fail(h, SR_OT_EUNSUPPORTED, "instance %d: permuted order in a batch needs m <= 2048", k);
        inst[k] = BatchInst{m[k], n[k], off_X[k], off_Y[k], off_a[k], off_b[k], off_T[k], atoms_total};
        atoms_total += (long long)m[k] * kAtomRecord;
        const int bk = bucket_of(n[k]);
        if (bk < 0) solo.push_back(k);
        else buckets[bk].push_back(k);
    }
    for (auto &bq : buckets)
        std::stable_sort(bq.begin(), bq.end(), [&](int x, int y) {
            return (long long)m[x] * n[x] > (long long)m[y] * n[y];
        });
    BatchInst *d_inst;
    int *d_queue, *d_head, *d_bad;
    BatchResult *d_res;
    int4 *d_atoms;
    if ((st = ws_typed(h, WS_B_INST, (size_t)batch, &d_inst))) return st;
    if ((st = ws_typed(h, WS_B_QUEUE, (size_t)batch, &d_queue))) return st;
    if ((st = ws_typed(h, WS_B_HEAD, (size_t)kNumBuckets, &d_head))) return st;
    if ((st = ws_typed(h, WS_B_RES, (size_t)batch, &d_res))) return st;
    if ((st = ws_typed(h, WS_B_BAD, (size_t)batch, &d_bad))) return st;
    if ((st = ws_typed(h, WS_B_ATOMS, (size_t)std::max(atoms_total, 1LL), &d_atoms))) return st;
    std::vector<int> queue;
    std::vector<int> qstart(kNumBuckets + 1, 0);
    for (int bk = 0; bk < kNumBuckets; ++bk) {
        qstart[bk] = (int)queue.size();
        queue.insert(queue.end(), buckets[bk].begin(), buckets[bk].end());
    }
    qstart[kNumBuckets] = (int)queue.size();
    CK(h, cudaMemcpyAsync(d_inst, inst.data(), sizeof(BatchInst) * batch, cudaMemcpyHostToDevice, h->stream));
    if (!queue.empty())
        CK(h, cudaMemcpyAsync(d_queue, queue.data(), sizeof(int) * queue.size(), cudaMemcpyHostToDevice, h->stream));
    // ---- input checks ------------------------------------------------------
    CK(h, cudaMemsetAsync(d_bad, 0, sizeof(int) * batch, h->stream));
    k_batch_check<<<std::min(batch, 152 * 4), 256, 0, h->stream>>>(d_inst, batch, X, Y, a, b, d_bad);
    h->launches += 1;
    CKL(h);
    {
        std::vector<int> bad(batch);
        CK(h, cudaMemcpyAsync(bad.data(), d_bad, sizeof(int) * batch, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        for (int k = 0; k < batch; ++k)
            if (bad[k]) return fail(h, SR_OT_EINVAL, "instance %d: %d negative or non-finite entries in a, b, X or Y", k, bad[k]);
    }
    if ((st = ensure_side_streams(h))) return st;

    sr_ot_status worst = SR_OT_OK;
    auto account = [&](sr_ot_status s) {
        if (s < 0 && (worst >= 0 || s < worst)) worst = s;
        else if (s == SR_OT_NOT_CONVERGED && worst == SR_OT_OK) worst = s;
    };
    // dense or oversize instances one at a time: from T0, or (warm start)
    // from the plan in T, which the batched kernels left feasible wherever
    // they stopped
    auto solve_solo = [&](const std::vector<int> &list, auto in_batch_width) {
        for (int k : list) {
            sr_ot_options o1 = *o;
            o1.dense_only = in_batch_width(k) ? 1 : o->dense_only;
            o1.trace = nullptr;
            o1.trace_capacity = 0;
            sr_ot_status s = solve_impl<float>(h, &o1, m[k], n[k], 3, nullptr, X + off_X[k], Y + off_Y[k],
                                               a + off_a[k], b + off_b[k], T + off_T[k],
                                               o->batch_warm_start ? 1 : 0, &res[k]);
            if (s < 0) res[k].status = s;
            account(s);
        }
    };
    // pairwise steps in cyclic or uniform order: the batched speculative form
    // (SR_OT_EPOCH_TWO_PHASE keeps the persistent two-phase kernel below)
    if (o->variant == SR_OT_BCPFW && (o->order == SR_OT_CYCLIC || o->order == SR_OT_UNIFORM) &&
        o->epoch_kernel != SR_OT_EPOCH_TWO_PHASE) {
        std::vector<int> rest;
        if ((st = solve_batched_spec(h, o, batch, m, n, inst, d_inst, d_atoms, X, Y, a, b, T, res, rest)))
            return st;
        std::vector<char> again(batch, 0);
        for (int k : rest) again[k] = 1;
        for (int k = 0; k < batch; ++k)
            if (!again[k]) account((sr_ot_status)res[k].status);
        solve_solo(rest, [&](int k) { return spec_batch_bucket(n[k]) >= 0; });
        return worst;
    }

    BatchArgs base;
    base.inst = d_inst;
    base.X = X;
    base.Y = Y;
    base.a = a;
    base.b = b;
    base.T = T;
    base.atoms = d_atoms;
    base.res = d_res;
    base.rho = o->rho;
    base.tol = o->tol_rel_gap;
    base.max_epochs = o->max_epochs;
    base.gap_every = o->gap_every;
    base.variant = o->variant;
    base.order = o->order;
    base.step = o->step;
    base.seed = o->seed;
    base.warm = o->batch_warm_start ? 1 : 0;
    int sms = 152;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    auto args_for = [&](int bk, int tile) {
        BatchArgs B = base;
        B.queue = d_queue + qstart[bk];
        B.queue_len = qstart[bk + 1] - qstart[bk];
        B.queue_head = d_head + bk;
        return B;
    };
    auto grid_for = [&](int bk, int tile) {
        const int len = qstart[bk + 1] - qstart[bk];
        return std::max(1, std::min(len, sms * batch_tile_ctas_per_sm(tile)));
    };
    // ---- autotune the tile of each bucket (first call per bucket and rule) --
    for (int bk = 0; bk < kNumBuckets; ++bk) {
        if (buckets[bk].empty()) continue;
        const long long key = bk * 64 + o->variant * 8 + o->step;
        if (h->tuned_tile.count(key)) continue;
        int best = kBucketTiles[bk][0];
        // the timing runs write the plans: not with a warm start (the first
        // tile of the bucket is taken until a cold call has tuned it)
        if (kBucketTiles[bk].size() > 1 && !base.warm) {
            double best_rate = -1.0;
            for (int tile : kBucketTiles[bk]) {
                BatchArgs B = args_for(bk, tile);
                B.max_epochs = 1;
                B.tol = 0.0;
                B.gap_every = 1;
                cudaEvent_t e0 = prof_event(h), e1 = prof_event(h);
                CK(h, cudaMemsetAsync(d_head + bk, 0, sizeof(int), h->stream));
                CK(h, cudaEventRecord(e0, h->stream));
                launch_batched_tile(tile, B, grid_for(bk, tile), h->stream);
                h->launches += 1;
                CK(h, cudaEventRecord(e1, h->stream));
                CKL(h);
                CK(h, cudaStreamSynchronize(h->stream));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                h->event_pool.push_back(e0);
                h->event_pool.push_back(e1);
                long long upd = 0;
                for (int k : buckets[bk]) upd += m[k];
                const double rate = upd / std::max(1e-6, (double)ms);
                if (rate > best_rate) { best_rate = rate; best = tile; }
            }
        }
        if (!base.warm) h->tuned_tile[key] = best;
    }
    // ---- the solve: one graph per shape set ----------------------------------
    unsigned long long hsh = 1469598103934665603ULL;
    auto mix = [&](unsigned long long v) { hsh = (hsh ^ v) * 1099511628211ULL; };
    mix((unsigned long long)batch);
    for (int k = 0; k < batch; ++k) {
        mix((unsigned long long)m[k]); mix((unsigned long long)n[k]);
        mix((unsigned long long)off_X[k]); mix((unsigned long long)off_Y[k]); mix((unsigned long long)off_a[k]);
        mix((unsigned long long)off_b[k]); mix((unsigned long long)off_T[k]);
    }
    mix((uintptr_t)X); mix((uintptr_t)Y); mix((uintptr_t)a); mix((uintptr_t)b); mix((uintptr_t)T);
    mix((uintptr_t)d_inst); mix((uintptr_t)d_atoms); mix((uintptr_t)d_res);
    mix((uintptr_t)d_queue); mix((uintptr_t)d_head);
    unsigned long long ob[8];
    std::memcpy(ob, o, std::min(sizeof(ob), sizeof(*o)));
    for (unsigned long long w : ob) mix(w);
    mix((unsigned long long)base.warm);
    for (int bk = 0; bk < kNumBuckets; ++bk) {  // the tile each bucket runs with
        auto tt = h->tuned_tile.find(bk * 64 + o->variant * 8 + o->step);
        mix(tt == h->tuned_tile.end() ? 99ull : (unsigned long long)tt->second);
    }
    cudaGraphExec_t exec = nullptr;
    auto it = h->graphs.find(hsh);
    if (it != h->graphs.end()) {
        exec = it->second;
    } else {
        // Captured on the handle's own stream (capture is not allowed on the
        // legacy default stream); the graph is then launched on the caller's.
        cudaGraph_t graph;
        cudaStream_t origin = h->side[0];
        CK(h, cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(d_head, 0, sizeof(int) * kNumBuckets, origin);
        cudaEventRecord(h->ev_fork, origin);
        int used = 0;
        for (int bk = 0; bk < kNumBuckets; ++bk) {
            if (buckets[bk].empty()) continue;
            auto tt = h->tuned_tile.find(bk * 64 + o->variant * 8 + o->step);
            const int tile = tt == h->tuned_tile.end() ? kBucketTiles[bk][0] : tt->second;
            cudaStream_t s = h->side[used];
            if (used > 0) cudaStreamWaitEvent(s, h->ev_fork, 0);
            launch_batched_tile(tile, args_for(bk, tile), grid_for(bk, tile), s);
            if (used > 0) cudaEventRecord(h->ev_join[used], s);
            ++used;
        }
        for (int k = 1; k < used; ++k) cudaStreamWaitEvent(origin, h->ev_join[k], 0);
        cudaError_t ce = cudaStreamEndCapture(origin, &graph);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return fail(h, SR_OT_ECUDA, "graph capture of the batched solve failed: %s", cudaGetErrorString(ce));
        }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return fail(h, SR_OT_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
        }
        h->graphs[hsh] = exec;
    }
    {
        ProfScope ps(h, SR_OT_PROF_BATCH);
        CK(h, cudaGraphLaunch(exec, h->stream));
    }
    int nlaunch = 0;
    for (int bk = 0; bk < kNumBuckets; ++bk) nlaunch += !buckets[bk].empty();
    h->launches += nlaunch;
    std::vector<BatchResult> hres(batch);
    CK(h, cudaMemcpyAsync(hres.data(), d_res, sizeof(BatchResult) * batch, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    prof_collect(h);
    // ---- fill results; dense or oversize instances one at a time ------------
    for (int k = 0; k < batch; ++k) {
        if (bucket_of(n[k]) < 0) continue;
        const BatchResult &r = hres[k];
        sr_ot_result &o2 = res[k];
        o2.objective = r.f;
        o2.gap = r.g;
        o2.rel_gap = r.f != 0.0 ? r.g / r.f : 0.0;
        o2.dual = r.f - r.g;
        o2.row_err = r.feas;
        o2.epochs = r.epochs;
        o2.block_updates = r.updates;
        o2.reserved = 0;
        o2.status = r.status == kInstOk ? SR_OT_OK
                  : r.status == kInstNotConverged ? SR_OT_NOT_CONVERGED
                  : r.status == kInstNonFinite ? SR_OT_ENUMERIC : SR_OT_OK;
        if (r.status == kInstNeedsDense) solo.push_back(k);
        else account((sr_ot_status)o2.status);
    }
    solve_solo(solo, [&](int k) { return bucket_of(n[k]) >= 0; });
    return worst;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void sr_ot_default_options(sr_ot_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->variant = SR_OT_BCFW;
    o->order = SR_OT_CYCLIC;
    o->step = SR_OT_DEC;
    o->precision = SR_OT_FP32;
    o->rho = 10.0;
    o->tol_rel_gap = 0.0;
    o->max_epochs = 100;
    o->gap_every = 1;
    o->refresh_every = 1;
    o->ga_M = 1;
    o->ga_global_only = 0;
    o->seed = 0;
    o->trace = nullptr;
    o->trace_capacity = 0;
    o->spin_limit = 0;
    o->start_gate = nullptr;
}

sr_ot_status sr_ot_create(sr_ot_handle *out, int device, void *cuda_stream) {
    if (!out) return fail(nullptr, SR_OT_EINVAL, "sr_ot_create: out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(nullptr, SR_OT_ECUDA, "no CUDA device available: %s", cudaGetErrorString(e));
    }
    if (device < 0 || device >= count) return fail(nullptr, SR_OT_EINVAL, "device %d out of range", device);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, SR_OT_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    sr_ot_ctx *h = new sr_ot_ctx();
    h->device = device;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMallocHost(&h->h_cert, kCertCount * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&h->h_status, 2 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&h->h_check, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        sr_ot_destroy(h);
        return fail(nullptr, SR_OT_ENOMEM, "pinned host buffer allocation failed");
    }
    *out = h;
    return SR_OT_OK;
}

sr_ot_status sr_ot_set_stream(sr_ot_handle h, void *cuda_stream) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return SR_OT_OK;
}

sr_ot_status sr_ot_destroy(sr_ot_handle h) {
    if (!h) return SR_OT_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    for (auto &b : h->ws)
        if (b.p) cudaFree(b.p);
    if (h->h_cert) cudaFreeHost(h->h_cert);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->h_check) cudaFreeHost(h->h_check);
    for (auto &p : h->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second);
    for (int k = 0; k < 4; ++k) {
        if (h->side[k]) cudaStreamDestroy(h->side[k]);
        if (h->ev_join[k]) cudaEventDestroy(h->ev_join[k]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    delete h;
    return SR_OT_OK;
}

const char *sr_ot_last_error(sr_ot_handle h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

sr_ot_status sr_ot_solve(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d,
                         const void *C, const void *X, const void *Y, const void *a, const void *b,
                         void *T_inout, int warm_start, sr_ot_result *res) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    sr_ot_status st;
    if ((st = check_opts(h, opts))) return st;
    if ((st = check_sizes(h, m, n))) return st;
    if (!a || !b || !T_inout) return fail(h, SR_OT_EINVAL, "a, b and T must be non-NULL");
    if ((st = check_stream_device(h))) return st;
    if (opts->precision == SR_OT_FP64)
        return solve_impl<double>(h, opts, m, n, d, C, X, Y, a, b, T_inout, warm_start, res);
    return solve_impl<float>(h, opts, m, n, d, C, X, Y, a, b, T_inout, warm_start, res);
}

sr_ot_status sr_ot_gap(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d,
                       const void *C, const void *X, const void *Y, const void *a, const void *b,
                       const void *T, double *g_rows, sr_ot_result *res) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    sr_ot_status st;
    if (!opts) return fail(h, SR_OT_EINVAL, "opts is NULL");
    if (!std::isfinite(opts->rho) || opts->rho < 0.0) return fail(h, SR_OT_EINVAL, "rho must be finite and >= 0");
    if ((st = check_sizes(h, m, n))) return st;
    if (!a || !b || !T) return fail(h, SR_OT_EINVAL, "a, b and T must be non-NULL");
    if ((st = check_stream_device(h))) return st;
    if (opts->precision == SR_OT_FP64)
        return gap_impl<double>(h, opts, m, n, d, C, X, Y, a, b, T, g_rows, res);
    return gap_impl<float>(h, opts, m, n, d, C, X, Y, a, b, T, g_rows, res);
}

sr_ot_status sr_ot_lp_metrics(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d, const void *C,
                              const void *X, const void *Y, const void *T, const void *T_lp,
                              sr_ot_lp_metrics_result *out) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    sr_ot_status st;
    if (!opts) return fail(h, SR_OT_EINVAL, "opts is NULL");
    if ((st = check_sizes(h, m, n))) return st;
    if (!T || !T_lp || !out) return fail(h, SR_OT_EINVAL, "T, T_lp and out must be non-NULL");
    const bool have_c = C != nullptr, have_pts = X != nullptr || Y != nullptr;
    if (have_c == have_pts) return fail(h, SR_OT_EINVAL, "pass exactly one of C or (X, Y)");
    if (have_pts && (!X || !Y)) return fail(h, SR_OT_EINVAL, "points mode needs both X and Y");
    if (have_pts && d != 3) return fail(h, SR_OT_EUNSUPPORTED, "the metrics take points with d = 3 (got %d); pass C", d);
    if (opts->cost_kind != SR_OT_COST_SQUARED && opts->cost_kind != SR_OT_COST_EUCLIDEAN)
        return fail(h, SR_OT_EINVAL, "unknown cost_kind %d", opts->cost_kind);
    if ((st = check_stream_device(h))) return st;
    const int nb = lp_metrics_blocks(m);
    double *wk;
    if ((st = ws_typed(h, WS_MET, (size_t)4 * nb + 4, &wk))) return st;
    {
        ProfScope ps(h, SR_OT_PROF_METRICS);
        if (opts->precision == SR_OT_FP64) {
            LpMetricsArgs<double> A{m, n, static_cast<const double *>(T), static_cast<const double *>(T_lp),
                                    static_cast<const double *>(C), static_cast<const double *>(X),
                                    static_cast<const double *>(Y), opts->cost_kind == SR_OT_COST_EUCLIDEAN};
            launch_lp_metrics<double>(A, wk, wk + 4 * nb, h->stream);
        } else {
            LpMetricsArgs<float> A{m, n, static_cast<const float *>(T), static_cast<const float *>(T_lp),
                                   static_cast<const float *>(C), static_cast<const float *>(X),
                                   static_cast<const float *>(Y), opts->cost_kind == SR_OT_COST_EUCLIDEAN};
            launch_lp_metrics<float>(A, wk, wk + 4 * nb, h->stream);
        }
    }
    h->launches += 2;
    CKL(h);
    CK(h, cudaMemcpyAsync(h->h_check, wk + 4 * nb, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    prof_collect(h);
    const double d2 = h->h_check[0], l2 = h->h_check[1], tc = h->h_check[2], lc = h->h_check[3];
    out->diff_norm = std::sqrt(std::max(d2, 0.0));
    out->lp_norm = std::sqrt(std::max(l2, 0.0));
    out->value = tc;
    out->lp_value = lc;
    out->e_m = out->lp_norm > 0.0 ? out->diff_norm / out->lp_norm : 0.0;
    out->e_v = lc != 0.0 ? std::fabs(tc - lc) / std::fabs(lc) : 0.0;
    return SR_OT_OK;
}

sr_ot_status sr_ot_solve_batched(sr_ot_handle h, const sr_ot_options *opts, int batch, const int *m,
                                 const int *n, int d, const long long *off_X, const long long *off_Y,
                                 const long long *off_a, const long long *off_b,
                                 const long long *off_T, const void *X, const void *Y, const void *a,
                                 const void *b, void *T, sr_ot_result *res) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    sr_ot_status st;
    if ((st = check_opts(h, opts))) return st;
    if ((st = check_stream_device(h))) return st;
    return solve_batched_impl(h, opts, batch, m, n, d, off_X, off_Y, off_a, off_b, off_T,
                              static_cast<const float *>(X), static_cast<const float *>(Y),
                              static_cast<const float *>(a), static_cast<const float *>(b),
                              static_cast<float *>(T), res);
}

sr_ot_status sr_ot_transfer(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d, const void *Y,
                            const void *a, const void *b, const void *T, void *Xhat, sr_ot_transfer_stats *stats) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    sr_ot_status st;
    if (!opts) return fail(h, SR_OT_EINVAL, "opts is NULL");
    if ((st = check_sizes(h, m, n))) return st;
    if ((st = check_stream_device(h))) return st;
    const long long z = 0;
    double out[4] = {0.0, 0.0, 0.0, 0.0};
    double *so = stats ? out : nullptr;
    if (opts->precision == SR_OT_FP64)
        st = adjoint_impl<double>(h, opts, 1, &m, &n, d, &z, &z, &z, &z, &z, nullptr, Y, a, b, T, nullptr, nullptr,
                                  nullptr, nullptr, Xhat, so);
    else
        st = adjoint_impl<float>(h, opts, 1, &m, &n, d, &z, &z, &z, &z, &z, nullptr, Y, a, b, T, nullptr, nullptr,
                                 nullptr, nullptr, Xhat, so);
    if (st == SR_OT_OK && stats) {
        stats->row_err = out[0];
        stats->col_err = out[1];
        stats->e_c = out[2];
        stats->sparsity = out[3];
    }
    return st;
}

sr_ot_status sr_ot_grad(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d,
                        const void *X, const void *Y, const void *a, const void *b, const void *T,
                        void *dC, void *dX, void *dY, void *db) {
    (void)a;
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    sr_ot_status st;
    if (!opts) return fail(h, SR_OT_EINVAL, "opts is NULL");
    if ((st = check_sizes(h, m, n))) return st;
    if ((st = check_stream_device(h))) return st;
    const long long z = 0;
    if (opts->precision == SR_OT_FP64)
        return grad_impl<double>(h, opts, 1, &m, &n, d, &z, &z, &z, &z, X, Y, b, T, dC, dX, dY, db);
    return grad_impl<float>(h, opts, 1, &m, &n, d, &z, &z, &z, &z, X, Y, b, T, dC, dX, dY, db);
}

sr_ot_status sr_ot_grad_batched(sr_ot_handle h, const sr_ot_options *opts, int batch, const int *m,
                                const int *n, int d, const long long *off_X, const long long *off_Y,
                                const long long *off_b, const long long *off_T, const void *X,
                                const void *Y, const void *b, const void *T, void *dX, void *dY,
                                void *db) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    sr_ot_status st;
    if (batch <= 0) return fail(h, SR_OT_EINVAL, "batch must be >= 1");
    if (!m || !n || !off_X || !off_Y || !off_b || !off_T)
        return fail(h, SR_OT_EINVAL, "size and offset arrays must be non-NULL");
    if ((st = check_stream_device(h))) return st;
    if (opts && opts->precision == SR_OT_FP64)
        return grad_impl<double>(h, opts, batch, m, n, d, off_X, off_Y, off_b, off_T, X, Y, b, T, nullptr,
                                 dX, dY, db);
    return grad_impl<float>(h, opts, batch, m, n, d, off_X, off_Y, off_b, off_T, X, Y, b, T, nullptr, dX,
                            dY, db);
}

sr_ot_status sr_ot_transfer_batched(sr_ot_handle h, const sr_ot_options *opts, int batch, const int *m,
                                    const int *n, int d, const long long *off_X, const long long *off_Y,
                                    const long long *off_a, const long long *off_b, const long long *off_T,
                                    const void *Y, const void *a, const void *b, const void *T, void *Xhat,
                                    sr_ot_transfer_stats *stats) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    sr_ot_status st;
    if (!opts) return fail(h, SR_OT_EINVAL, "opts is NULL");
    if (batch <= 0) return fail(h, SR_OT_EINVAL, "batch must be >= 1");
    if (!m || !n || !off_X || !off_Y || !off_a || !off_b || !off_T)
        return fail(h, SR_OT_EINVAL, "size and offset arrays must be non-NULL");
    if ((st = check_stream_device(h))) return st;
    std::vector<double> out(stats ? 4 * (size_t)batch : 0);
    double *so = stats ? out.data() : nullptr;
    if (opts->precision == SR_OT_FP64)
        st = adjoint_impl<double>(h, opts, batch, m, n, d, off_X, off_Y, off_b, off_T, off_a, nullptr, Y, a, b, T,
                                  nullptr, nullptr, nullptr, nullptr, Xhat, so);
    else
        st = adjoint_impl<float>(h, opts, batch, m, n, d, off_X, off_Y, off_b, off_T, off_a, nullptr, Y, a, b, T,
                                 nullptr, nullptr, nullptr, nullptr, Xhat, so);
    if (st == SR_OT_OK && stats)
        for (int k = 0; k < batch; ++k) {
            stats[k].row_err = out[4 * k];
            stats[k].col_err = out[4 * k + 1];
            stats[k].e_c = out[4 * k + 2];
            stats[k].sparsity = out[4 * k + 3];
        }
    return st;
}

long long sr_ot_launch_count(sr_ot_handle h) { return h ? h->launches : 0; }

sr_ot_status sr_ot_profile_chain_floor(sr_ot_handle h, int chain_warps, int updates, double *ns_per_update) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    h->err.clear();
    if (chain_warps != 1 && chain_warps != 3) return fail(h, SR_OT_EINVAL, "chain_warps must be 1 or 3");
    if (updates < 1 || !ns_per_update) return fail(h, SR_OT_EINVAL, "updates must be >= 1 and the output non-NULL");
    sr_ot_status st;
    if ((st = check_stream_device(h))) return st;
    int *wk;
    if ((st = ws_typed(h, WS_FLOOR, 4, &wk))) return st;
    CK(h, cudaMemsetAsync(wk, 0, sizeof(int), h->stream));
    cudaEvent_t e0 = prof_event(h), e1 = prof_event(h);
    CK(h, cudaEventRecord(e0, h->stream));
    launch_chain_floor(chain_warps, updates, wk, reinterpret_cast<float *>(wk + 1), h->stream);
    h->launches += 1;
    CK(h, cudaEventRecord(e1, h->stream));
    CKL(h);
    CK(h, cudaMemcpyAsync(h->h_status, wk, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->event_pool.push_back(e0);
    h->event_pool.push_back(e1);
    if (h->h_status[0]) return dev_status_error(h, h->h_status[0]);
    *ns_per_update = 1e6 * (double)ms / (double)updates;
    return SR_OT_OK;
}

sr_ot_status sr_ot_profile_enable(sr_ot_handle h, int enable) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    cudaStreamSynchronize(h->stream);
    prof_collect(h);
    h->prof = enable != 0;
    for (int k = 0; k < SR_OT_PROF_KINDS; ++k) { h->prof_ms[k] = 0.0; h->prof_groups[k] = 0; }
    return SR_OT_OK;
}

sr_ot_status sr_ot_profile_read(sr_ot_handle h, int kind, double *total_ms, long long *groups) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    if (kind < 0 || kind >= SR_OT_PROF_KINDS) return fail(h, SR_OT_EINVAL, "unknown profile class %d", kind);
    CK(h, cudaStreamSynchronize(h->stream));
    prof_collect(h);
    if (total_ms) *total_ms = h->prof_ms[kind];
    if (groups) *groups = h->prof_groups[kind];
    return SR_OT_OK;
}

sr_ot_status sr_ot_cost_bf16(sr_ot_handle h, int m, int n, int d, const float *X, const float *Y,
                             float *C) {
    if (!h) return fail(nullptr, SR_OT_EINVAL, "handle is NULL");
    sr_ot_status st;
    if ((st = check_sizes(h, m, n))) return st;
    if (!X || !Y || !C) return fail(h, SR_OT_EINVAL, "X, Y and C must be non-NULL");
    if ((st = check_stream_device(h))) return st;
    void *ws;
    int *err;
    if ((st = ws_get(h, WS_BF16, cost_bf16_workspace(m, n, d), &ws))) return st;
    if ((st = ws_typed(h, WS_BF16_ERR, 1, &err))) return st;
    CK(h, cudaMemsetAsync(err, 0, sizeof(int), h->stream));
    const char *msg;
    {
        ProfScope ps(h, SR_OT_PROF_COST);
        msg = launch_cost_bf16(m, n, d, X, Y, C, ws, err, h->stream);
    }
    if (msg) return fail(h, SR_OT_EUNSUPPORTED, "BF16 cost: %s", msg);
    h->launches += 2;  // rounding, GEMM
    CKL(h);
    CK(h, cudaMemcpyAsync(h->h_status, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->h_status[0]) return fail(h, SR_OT_ETIMEOUT, "BF16 cost: a bounded device wait gave up");
    return SR_OT_OK;
}

}  // extern "C"
