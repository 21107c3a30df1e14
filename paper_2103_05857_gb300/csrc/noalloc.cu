// noalloc.cu -- sr_ot_gap_noalloc: the duality-gap certificate without any
// memory allocation.
//
// Some callers cannot allocate device memory at the point where they want a
// certificate: an application whose caching allocator has reserved the
// device's memory up front, a plug-in embedded in a host program that owns
// every allocation, a long-running service that must not fail on
// fragmentation after start-up. This entry point serves them: it takes no
// handle (creating one allocates a workspace and a pinned result buffer) and
// runs the certificate kernels on a fixed scratch area that lives in this
// file as a static __device__ array, so it is part of the module image and
// exists on every device that loads the library, until the process exits.
// The call synchronises its stream before it returns (it reads the input
// checks and the certificate back to the host).
//
// Limits: scratch is kNoAllocScratchBytes. The certificate's column sums are
// taken in row chunks; when the default chunking does not fit, one chunk is
// used (the column sums are then summed over all rows in one pass, which is
// slower but needs n doubles only). Sizes that do not fit even then are
// rejected with SR_OT_EUNSUPPORTED. With 4 MiB every n <= 207,552 fits for
// any m (the bound is reached for m >= 9,721, where the row pass uses its
// largest grid); smaller m leave room for slightly larger n.
// The cost must be given (C) or come from d = 3 points (no materialised cost
// for other d, no BF16 tensor-core cost).
//
// Sharing: every call uses the same array and leaves the last call's values
// in it. Calls whose kernels overlap on the GPU (different streams or
// threads without ordering between them) race on it; serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/sr_ot.h"
#include "common.cuh"
#include "internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 4u << 20;  // 4 MiB per device
constexpr int kMaxDevices = 64;

// The scratch area. In host code this name is only a stand-in for the
// device symbol; host code uses the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Errors are reported through sr_ot_last_error(NULL), like sr_ot_create's.
sr_ot_status nfail(sr_ot_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    srot::set_handleless_error(buf);
    return st;
}

// Device address of the scratch array on `device` (current device), looked
// up once per device.
sr_ot_status scratch_address(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return nfail(SR_OT_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return nfail(SR_OT_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                         cudaGetErrorString(e));
        }
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return SR_OT_OK;
}

size_t rounded(size_t bytes);

// Bytes of scratch that a certificate plan `w` of an m x n instance takes.
size_t scratch_need(const srot::CertWork &w, int n);

// Restores the calling thread's current device when it goes out of scope.
struct DeviceGuard {
    int saved = -1;
    ~DeviceGuard() {
        if (saved >= 0) cudaSetDevice(saved);
    }
};

template <typename T>
T *carve(unsigned char *&cur, size_t count) {
    T *p = reinterpret_cast<T *>(cur);
    cur += ((count * sizeof(T) + 255) / 256) * 256;
    return p;
}

size_t rounded(size_t bytes) { return ((bytes + 255) / 256) * 256; }

size_t scratch_need(const srot::CertWork &w, int n) {
    return rounded((size_t)w.nchunks * n * sizeof(double)) + rounded((size_t)n * sizeof(double)) +
           rounded((size_t)n * sizeof(float)) + rounded((size_t)2 * w.ncolblocks * sizeof(double)) +
           rounded((size_t)3 * w.nrowblocks * sizeof(double)) + rounded(srot::kCertCount * sizeof(double)) +
           rounded(4 * sizeof(int));
}

template <typename Real>
__global__ void k_noalloc_check(int m, int n, const Real *a, const Real *b, const Real *src,
                                long long nsrc, const Real *src2, long long nsrc2, int *bad) {
    int c0 = 0, c1 = 0, c2 = 0;
    long long tot = m;
    if (n > tot) tot = n;
    if (nsrc > tot) tot = nsrc;
    if (nsrc2 > tot) tot = nsrc2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < m) c0 += !(isfinite((double)a[e]) && a[e] >= Real(0));
        if (e < n) c1 += !(isfinite((double)b[e]) && b[e] >= Real(0));
        if (e < nsrc) c2 += !isfinite((double)src[e]);
        if (e < nsrc2) c2 += !isfinite((double)src2[e]);
    }
    if (c0) atomicAdd(&bad[0], c0);
    if (c1) atomicAdd(&bad[1], c1);
    if (c2) atomicAdd(&bad[2], c2);
}

template <typename Real>
sr_ot_status gap_noalloc(int device, cudaStream_t st, const sr_ot_options *o, int m, int n, int d,
                         const void *C, const void *X, const void *Y, const void *a, const void *b,
                         const void *T, double *g_rows, sr_ot_result *res) {
    using namespace srot;
    Inst<Real> in;
    in.m = m;
    in.n = n;
    in.a = static_cast<const Real *>(a);
    in.b = static_cast<const Real *>(b);
    in.C = static_cast<const Real *>(C);
    in.X = static_cast<const Real *>(X);
    in.Y = static_cast<const Real *>(Y);
    const bool have_c = C != nullptr, have_pts = X != nullptr || Y != nullptr;
    if (have_c == have_pts) return nfail(SR_OT_EINVAL, "pass exactly one of C or (X, Y)");
    if (have_pts) {
        if (!X || !Y) return nfail(SR_OT_EINVAL, "points mode needs both X and Y");
        if (d != 3) return nfail(SR_OT_EINVAL, "the no-allocation certificate takes points with d = 3 only (got d = %d)", d);
        in.cost_mode = kCostPts3;
    } else {
        in.cost_mode = kCostGiven;
    }

    CertWork w;
    cert_work_shape(m, n, &w.nchunks, &w.rows_per_chunk, &w.ncolblocks, &w.nrowblocks);
    if (scratch_need(w, n) > kNoAllocScratchBytes) {
        // one row chunk: the column partials shrink to n doubles
        w.nchunks = 1;
        w.rows_per_chunk = std::max(8, m);
    }
    const size_t need = scratch_need(w, n);
    if (need > kNoAllocScratchBytes)
        return nfail(SR_OT_EUNSUPPORTED,
                     "m = %d, n = %d needs %zu bytes of certificate scratch; the no-allocation entry point has %zu",
                     m, n, need, kNoAllocScratchBytes);

    unsigned char *base = nullptr;
    sr_ot_status s = scratch_address(device, &base);
    if (s != SR_OT_OK) return s;
    unsigned char *cur = base;
    w.partial = carve<double>(cur, (size_t)w.nchunks * n);
    w.r64 = carve<double>(cur, n);
    w.rq32 = carve<float>(cur, n);
    w.colpart = carve<double>(cur, (size_t)2 * w.ncolblocks);
    w.rowpart = carve<double>(cur, (size_t)3 * w.nrowblocks);
    w.cert = carve<double>(cur, kCertCount);
    int *bad = carve<int>(cur, 4);

    // input checks: the counters must start at zero on every call
    cudaError_t e = cudaMemsetAsync(bad, 0, 4 * sizeof(int), st);
    if (e != cudaSuccess) return nfail(SR_OT_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    const long long n1 = have_c ? (long long)m * n : (long long)m * 3;
    const long long n2 = have_c ? 0 : (long long)n * 3;
    const Real *s1 = have_c ? in.C : in.X;
    long long tot = std::max<long long>(std::max<long long>(m, n), std::max(n1, n2));
    int blocks = (int)std::min<long long>((tot + 255) / 256, 152 * 8);
    k_noalloc_check<Real><<<blocks, 256, 0, st>>>(m, n, in.a, in.b, s1, n1, have_c ? nullptr : in.Y, n2, bad);
    int hbad[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return nfail(SR_OT_ECUDA, "input check: %s", cudaGetErrorString(e));
    if (hbad[0]) return nfail(SR_OT_EINVAL, "a has %d negative or non-finite entries", hbad[0]);
    if (hbad[1]) return nfail(SR_OT_EINVAL, "b has %d negative or non-finite entries", hbad[1]);
    if (hbad[2]) return nfail(SR_OT_ENUMERIC, "cost input has %d non-finite entries", hbad[2]);

    launch_certificate<Real>(in, static_cast<const Real *>(T), o->rho, o->tol_rel_gap, w, nullptr,
                             g_rows, st);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return nfail(SR_OT_ECUDA, "certificate launch: %s", cudaGetErrorString(e));
    double cert[kCertCount];
    if ((e = cudaMemcpyAsync(cert, w.cert, sizeof(cert), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return nfail(SR_OT_ECUDA, "certificate: %s", cudaGetErrorString(e));
    if (res) {
        res->objective = cert[kCertF];
        res->gap = cert[kCertG];
        res->rel_gap = cert[kCertRel];
        res->dual = cert[kCertW];
        res->row_err = cert[kCertFeas];
        res->epochs = 0;
        res->block_updates = 0;
        res->status = SR_OT_OK;
        res->reserved = 0;
    }
    return SR_OT_OK;
}

}  // namespace

extern "C" {

sr_ot_status sr_ot_gap_noalloc(int device, void *cuda_stream, const sr_ot_options *opts, int m, int n,
                               int d, const void *C, const void *X, const void *Y, const void *a,
                               const void *b, const void *T, double *g_rows, sr_ot_result *res) {
    srot::set_handleless_error("");
    if (!opts) return nfail(SR_OT_EINVAL, "opts is NULL");
    if (!std::isfinite(opts->rho) || opts->rho < 0.0) return nfail(SR_OT_EINVAL, "rho must be finite and >= 0");
    if (m <= 0 || n <= 0) return nfail(SR_OT_EINVAL, "m and n must be >= 1 (got m=%d, n=%d)", m, n);
    if (!a || !b || !T) return nfail(SR_OT_EINVAL, "a, b and T must be non-NULL");
    if (opts->precision == SR_OT_FP32_BF16COST)
        return nfail(SR_OT_EINVAL, "the no-allocation certificate takes SR_OT_FP64 or SR_OT_FP32");
    if ((X || Y) && opts->cost_kind != SR_OT_COST_SQUARED)
        return nfail(SR_OT_EUNSUPPORTED, "the no-allocation certificate builds the squared cost from points only "
                                         "(pass the Euclidean cost as C)");
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(SR_OT_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    DeviceGuard guard;  // the caller's current device is restored on every return
    if (cur != device) {
        if ((e = cudaSetDevice(device)) != cudaSuccess) {
            cudaGetLastError();
            return nfail(SR_OT_ECUDA, "cudaSetDevice(%d): %s", device, cudaGetErrorString(e));
        }
        guard.saved = cur;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (opts->precision == SR_OT_FP64)
        return gap_noalloc<double>(device, st, opts, m, n, d, C, X, Y, a, b, T, g_rows, res);
    return gap_noalloc<float>(device, st, opts, m, n, d, C, X, Y, a, b, T, g_rows, res);
}

}  // extern "C"
