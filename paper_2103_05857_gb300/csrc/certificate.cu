// certificate.cu -- duality-gap certificate of a plan (Thm 2), initial plan
// and residual, per-epoch block permutation, plain cost materialisation.
//
// Certificate (Thm 2, eq. 11), in the library's orientation (rows = blocks):
//   s = T^T 1, r = s - b, grad_ij = C_ij + rho r_j,
//   f = <C,T> + (rho/2)||r||^2,
//   g = sum_i [ <t_i, grad_i> - a_i min_j grad_ij ]
//     = <C,T> + rho <s, r> - sum_i a_i min_j grad_ij,
//   w = f - g (the Lagrangian dual value, App. D).
// Two HBM passes over T: column sums (pass 1), then one warp per row for the
// row minimum and <t_i, c_i> (pass 2); every reduction is in a fixed order,
// so the result is bitwise reproducible run to run.
//
// Precision. FP64 plans are summed in double. FP32 plans are summed with
// compensated FP32 (Kahan, TwoProduct for t*c) and combined in double; the
// row argmin is taken on FP32 gradients and the minimum re-evaluated in
// double at the chosen column, so the computed gap can exceed the exact one
// by at most one FP32 rounding of the gradient per row and never under-states
// a row's distance from its LMO vertex by more than that.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace srot {

constexpr int kColThreads = 256;
constexpr int kRowThreads = 256;
constexpr int kRowWarps = kRowThreads / kWarp;
constexpr int kFinalThreads = 256;

void cert_work_shape(int m, int n, int *nchunks, int *rows_per_chunk, int *ncolblocks,
                     int *nrowblocks) {
    int colb = ceil_div(n, kColThreads);
    int target = 152 * 8;
    int chunks = std::max(1, std::min(m, target / std::max(1, colb)));
    int rpc = std::max(8, ceil_div(m, chunks));
    *rows_per_chunk = rpc;
    *nchunks = std::max(1, ceil_div(m, rpc));
    *ncolblocks = colb;
    *nrowblocks = std::max(1, std::min(ceil_div(m, kRowWarps), 152 * 8));
}

template <typename Real>
__device__ inline Real cost_at(const Inst<Real> &in, int i, int j);

template <>
__device__ inline float cost_at<float>(const Inst<float> &in, int i, int j) {
    if (in.cost_mode == kCostGiven) return in.C[(size_t)i * in.n + j];
    const float *x = in.X + (size_t)i * 3;
    const float *y = in.Y + (size_t)j * 3;
    float d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    return fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0)));
}

template <>
__device__ inline double cost_at<double>(const Inst<double> &in, int i, int j) {
    if (in.cost_mode == kCostGiven) return in.C[(size_t)i * in.n + j];
    const double *x = in.X + (size_t)i * 3;
    const double *y = in.Y + (size_t)j * 3;
    double d0 = dsub(x[0], y[0]), d1 = dsub(x[1], y[1]), d2 = dsub(x[2], y[2]);
    return dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2));
}

// ---------------------------------------------------------------------------
// Pass 1: column sums over a chunk of rows (ascending rows within a chunk).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kColThreads)
k_colsum_partial(const Real *__restrict__ T, int m, int n, int rpc, double *__restrict__ partial) {
    int j = blockIdx.x * kColThreads + threadIdx.x;
    int c = blockIdx.y;
    if (j >= n) return;
    int i0 = c * rpc, i1 = min(m, i0 + rpc);
    const Real *p = T + (size_t)i0 * n + j;
    if constexpr (std::is_same<Real, float>::value) {
        Kahan32 acc;
#pragma unroll 8
        for (int i = i0; i < i1; ++i, p += n) acc.add(__ldg(p));
        partial[(size_t)c * n + j] = acc.value();
    } else {
        double s = 0.0;
#pragma unroll 8
        for (int i = i0; i < i1; ++i, p += n) s += __ldg(p);
        partial[(size_t)c * n + j] = s;
    }
}

// Deterministic block sum of two doubles; result valid in thread 0.
__device__ inline void block_sum2(double &x, double &y) {
    __shared__ double sh[2][32];
    x = warp_sum(x);
    y = warp_sum(y);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = x; sh[1][w] = y; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        x = l < nw ? sh[0][l] : 0.0;
        y = l < nw ? sh[1][l] : 0.0;
        x = warp_sum(x);
        y = warp_sum(y);
    }
    __syncthreads();
}

// Column sums across chunks (ascending chunks), residual, optional refresh
// of the solver's running residual, and per-block partials of ||r||^2, <s,r>.
template <typename Real>
__global__ void __launch_bounds__(kColThreads)
k_colsum_final(const double *__restrict__ partial, int nchunks, int n, const Real *__restrict__ b,
               double rho, double *__restrict__ r64, float *__restrict__ rq32, double *refresh_q,
               double *__restrict__ colpart) {
    int j = blockIdx.x * kColThreads + threadIdx.x;
    double rr = 0.0, sr = 0.0;
    if (j < n) {
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += partial[(size_t)c * n + j];
        double r = s - (double)b[j];
        r64[j] = r;
        rq32[j] = (float)(rho * r);
        if (refresh_q) {
            if constexpr (std::is_same<Real, float>::value) refresh_q[j] = rho * r;
            else refresh_q[j] = r;
        }
        rr = r * r;
        sr = s * r;
    }
    block_sum2(rr, sr);
    if (threadIdx.x == 0) {
        colpart[2 * blockIdx.x + 0] = rr;
        colpart[2 * blockIdx.x + 1] = sr;
    }
}

// ---------------------------------------------------------------------------
// Pass 2: one warp per row: argmin of the row gradient, <t_i, c_i>,
// and the per-row gap.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kRowThreads)
k_gap_rows(Inst<Real> in, const Real *__restrict__ T, double rho, const double *__restrict__ r64,
           const float *__restrict__ rq32, double *__restrict__ g_rows, double *__restrict__ rowpart,
           int *__restrict__ js_out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = in.n;
    double acc_tc = 0.0, acc_amin = 0.0, acc_feas = 0.0;  // lane 0 of each warp accumulates its rows
    for (int i = blockIdx.x * kRowWarps + warp; i < in.m; i += gridDim.x * kRowWarps) {
        const Real *ti = T + (size_t)i * n;
        double tc_row, tr_row, rs_row;
        int jb;
        if constexpr (std::is_same<Real, float>::value) {
            Kahan32 tc, tr, rs;
            float tc_err = 0.f;
            uint32_t kb = 0xFFFFFFFFu;
            jb = 0x7FFFFFFF;
            if (in.cost_mode == kCostGiven) {
                // given C: kU columns per lane per step, their loads issued
                // before any is used (the columns are still visited in
                // ascending order); on-the-fly costs measured faster unbatched
                constexpr int kU = 4;
                for (int jb0 = 0; jb0 < n; jb0 += kU * kWarp) {
                    float tv[kU], cv[kU], qv[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int j = jb0 + u * kWarp + lane;
                        const bool ok = j < n;
                        tv[u] = ok ? __ldg(ti + j) : 0.f;
                        cv[u] = ok ? cost_at<float>(in, i, j) : 0.f;
                        qv[u] = ok ? __ldg(rq32 + j) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int j = jb0 + u * kWarp + lane;
                        const float t = tv[u], c = cv[u];
                        uint32_t k = f2key(c + qv[u]);
                        if (j < n && (k < kb || jb == 0x7FFFFFFF)) { kb = k; jb = j; }
                        if (t != 0.f) {
                            rs.add(t);
                            float p = __fmul_rn(t, c);
                            tc_err += fmaf(t, c, -p);  // exact rounding error of p (TwoProduct)
                            tc.add(p);
                            tr.add(__fmul_rn(t, (float)__ldg(r64 + j)));
                        }
                    }
                }
            } else {
                for (int j = lane; j < n; j += kWarp) {
                    float t = __ldg(ti + j);
                    float c = cost_at<float>(in, i, j);
                    uint32_t k = f2key(c + __ldg(rq32 + j));
                    if (k < kb || jb == 0x7FFFFFFF) { kb = k; jb = j; }
                    if (t != 0.f) {
                        rs.add(t);
                        float p = __fmul_rn(t, c);
                        tc_err += fmaf(t, c, -p);  // exact rounding error of p (TwoProduct)
                        tc.add(p);
                        tr.add(__fmul_rn(t, (float)__ldg(r64 + j)));
                    }
                }
            }
            uint32_t wk = __reduce_min_sync(0xffffffffu, kb);
            jb = __reduce_min_sync(0xffffffffu, kb == wk ? jb : 0x7FFFFFFF);
            tc_row = warp_sum(tc.value() + (double)tc_err);
            tr_row = warp_sum(tr.value());
            rs_row = warp_sum(rs.value());
        } else {
            double tc = 0.0, tr = 0.0, gb = 0.0, rs = 0.0;
            jb = 0x7FFFFFFF;
            for (int j = lane; j < n; j += kWarp) {
                double t = __ldg(ti + j);
                double c = cost_at<double>(in, i, j);
                double g = dadd(c, dmul(rho, __ldg(r64 + j)));
                if (jb == 0x7FFFFFFF || g < gb) { gb = g; jb = j; }
                tc += t * c;
                tr += t * __ldg(r64 + j);
                rs += t;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double og = __shfl_xor_sync(0xffffffffu, gb, o);
                int oj = __shfl_xor_sync(0xffffffffu, jb, o);
                bool take = (oj != 0x7FFFFFFF) &&
                            (jb == 0x7FFFFFFF || og < gb || (og == gb && oj < jb));
                if (take) { gb = og; jb = oj; }
            }
            tc_row = warp_sum(tc);
            tr_row = warp_sum(tr);
            rs_row = warp_sum(rs);
        }
        if (lane == 0) {
            double ai = (double)in.a[i];
            // jb < n always holds for n >= 1 (every lane with a column sets it)
            double gmin = (jb >= 0 && jb < n) ? (double)cost_at<Real>(in, i, jb) + rho * r64[jb] : NAN;
            acc_tc += tc_row;
            acc_amin += ai * gmin;
            const double dfe = fabs(rs_row - ai) / (ai > 0.0 ? ai : 1e-300);
            acc_feas = fmax(acc_feas, dfe);
            if (g_rows) g_rows[i] = tc_row + rho * tr_row - ai * gmin;
            if (js_out) js_out[i] = jb;
        }
    }
    __shared__ double sh[3][kRowWarps];
    if (lane == 0) { sh[0][warp] = acc_tc; sh[1][warp] = acc_amin; sh[2][warp] = acc_feas; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < kRowWarps; ++w) { a0 += sh[0][w]; a1 += sh[1][w]; a2 = fmax(a2, sh[2][w]); }
        rowpart[3 * blockIdx.x + 0] = a0;
        rowpart[3 * blockIdx.x + 1] = a1;
        rowpart[3 * blockIdx.x + 2] = a2;
    }
}

__global__ void __launch_bounds__(kFinalThreads)
k_cert_final(const double *__restrict__ colpart, int ncol, const double *__restrict__ rowpart,
             int nrow, double rho, double tol, double *__restrict__ cert) {
    double rr = 0.0, sr = 0.0, tc = 0.0, am = 0.0, fe = 0.0;
    for (int k = threadIdx.x; k < ncol; k += kFinalThreads) {
        rr += colpart[2 * k];
        sr += colpart[2 * k + 1];
    }
    for (int k = threadIdx.x; k < nrow; k += kFinalThreads) {
        tc += rowpart[3 * k];
        am += rowpart[3 * k + 1];
        fe = fmax(fe, rowpart[3 * k + 2]);
    }
    block_sum2(rr, sr);
    block_sum2(tc, am);
    __shared__ double shf[32];
    for (int o = 16; o > 0; o >>= 1) fe = fmax(fe, __shfl_xor_sync(0xffffffffu, fe, o));
    if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = fe;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < kFinalThreads / 32; ++w) fe = fmax(fe, shf[w]);
        double lin = tc, pen = 0.5 * rho * rr;
        double f = lin + pen;
        double g = lin + rho * sr - am;
        cert[kCertF] = f;
        cert[kCertG] = g;
        cert[kCertW] = f - g;
        cert[kCertLin] = lin;
        cert[kCertPen] = pen;
        cert[kCertRel] = (f != 0.0) ? g / f : (g == 0.0 ? 0.0 : INFINITY);
        cert[kCertFeas] = fe;
        cert[kCertStop] = (tol > 0.0 && g <= tol * f && fe <= kFeasTol) ? 1.0 : 0.0;
    }
}

template <typename Real>
void launch_certificate(const Inst<Real> &in, const Real *T, double rho, double tol,
                        const CertWork &w, double *refresh_q, double *g_rows, cudaStream_t st,
                        int *js_out) {
    dim3 g1(ceil_div(in.n, kColThreads), w.nchunks);
    k_colsum_partial<Real><<<g1, kColThreads, 0, st>>>(T, in.m, in.n, w.rows_per_chunk, w.partial);
    k_colsum_final<Real><<<w.ncolblocks, kColThreads, 0, st>>>(w.partial, w.nchunks, in.n, in.b,
                                                               rho, w.r64, w.rq32, refresh_q,
                                                               w.colpart);
    k_gap_rows<Real><<<w.nrowblocks, kRowThreads, 0, st>>>(in, T, rho, w.r64, w.rq32, g_rows,
                                                           w.rowpart, js_out);
    k_cert_final<<<1, kFinalThreads, 0, st>>>(w.colpart, w.ncolblocks, w.rowpart, w.nrowblocks,
                                              rho, tol, w.cert);
}

template void launch_certificate<float>(const Inst<float> &, const float *, double, double,
                                        const CertWork &, double *, double *, cudaStream_t, int *);
template void launch_certificate<double>(const Inst<double> &, const double *, double, double,
                                         const CertWork &, double *, double *, cudaStream_t, int *);

// ---------------------------------------------------------------------------
// Initial plan T0 = (a_i e_0) (Thm 1) and the solver's initial residual.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_init_plan(int m, int n, const Real *__restrict__ a, Real *__restrict__ T) {
    size_t total = (size_t)m * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        size_t i = e / n, j = e - i * n;
        T[e] = (j == 0) ? a[i] : Real(0);
    }
}

// One thread per column, rows in ascending order with FP64 accumulation (the
// FP64 path reproduces the oracle's column sums bit for bit this way).
template <typename Real>
__global__ void k_init_residual(int m, int n, const Real *__restrict__ T, const Real *__restrict__ b,
                                double rho, double *__restrict__ q) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    const Real *p = T + j;
#pragma unroll 4
    for (int i = 0; i < m; ++i, p += n) s = dadd(s, (double)__ldg(p));
    if constexpr (std::is_same<Real, float>::value) q[j] = rho * (s - (double)b[j]);
    else q[j] = dsub(s, b[j]);
}

template <typename Real>
void launch_init_residual(const Inst<Real> &in, const Real *T, double rho, double *q,
                          cudaStream_t st) {
    k_init_residual<Real><<<ceil_div(in.n, 128), 128, 0, st>>>(in.m, in.n, T, in.b, rho, q);
}

template <typename Real>
void launch_init_plan(const Inst<Real> &in, Real *T, int warm, double rho, double *q,
                      cudaStream_t st) {
    if (!warm) {
        size_t total = (size_t)in.m * in.n;
        int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
        k_init_plan<Real><<<blocks, 256, 0, st>>>(in.m, in.n, in.a, T);
    }
    launch_init_residual<Real>(in, T, rho, q, st);
}

template void launch_init_plan<float>(const Inst<float> &, float *, int, double, double *, cudaStream_t);
template void launch_init_plan<double>(const Inst<double> &, double *, int, double, double *, cudaStream_t);
template void launch_init_residual<float>(const Inst<float> &, const float *, double, double *, cudaStream_t);
template void launch_init_residual<double>(const Inst<double> &, const double *, double, double *, cudaStream_t);

// ---------------------------------------------------------------------------
// Permutation of 0..m-1 for one epoch: positions sorted by the 64-bit key
// splitmix64(seed, stream 1, epoch*m + t), ties by index (bitonic sort).
// ---------------------------------------------------------------------------
constexpr int kPermSmemMax = 16384;

__device__ inline bool kv_less(uint64_t ka, int ia, uint64_t kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

__global__ void __launch_bounds__(1024)
k_perm_smem(unsigned long long seed, long long epoch, int m, int L, int *__restrict__ perm) {
    extern __shared__ unsigned char smem_raw[];
    uint64_t *key = reinterpret_cast<uint64_t *>(smem_raw);
    int *idx = reinterpret_cast<int *>(key + L);
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        if (t < m) {
            key[t] = sm64_draw(seed, 1, (uint64_t)epoch * (uint64_t)m + (uint64_t)t);
            idx[t] = t;
        } else {
            key[t] = ~0ULL;
            idx[t] = 0x7FFFFFFF;
        }
    }
    __syncthreads();
    for (int k = 2; k <= L; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < L; t += blockDim.x) {
                int l = t ^ j;
                if (l > t) {
                    bool up = (t & k) == 0;
                    uint64_t kt = key[t], kl = key[l];
                    int it = idx[t], il = idx[l];
                    bool sw = up ? kv_less(kl, il, kt, it) : kv_less(kt, it, kl, il);
                    if (sw) { key[t] = kl; key[l] = kt; idx[t] = il; idx[l] = it; }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < m; t += blockDim.x) perm[t] = idx[t];
}

__global__ void k_perm_fill(unsigned long long seed, long long epoch, int m, int L,
                            uint64_t *__restrict__ key, int *__restrict__ idx) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L) return;
    if (t < m) {
        key[t] = sm64_draw(seed, 1, (uint64_t)epoch * (uint64_t)m + (uint64_t)t);
        idx[t] = t;
    } else {
        key[t] = ~0ULL;
        idx[t] = 0x7FFFFFFF;
    }
}

__global__ void k_perm_step(int L, int j, int k, uint64_t *__restrict__ key, int *__restrict__ idx) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L) return;
    int l = t ^ j;
    if (l <= t) return;
    bool up = (t & k) == 0;
    uint64_t kt = key[t], kl = key[l];
    int it = idx[t], il = idx[l];
    bool sw = up ? kv_less(kl, il, kt, it) : kv_less(kt, it, kl, il);
    if (sw) { key[t] = kl; key[l] = kt; idx[t] = il; idx[l] = it; }
}

__global__ void k_perm_copy(int m, const int *__restrict__ idx, int *__restrict__ perm) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) perm[t] = idx[t];
}

static int next_pow2(int m) {
    int L = 1;
    while (L < m) L <<= 1;
    return L;
}

size_t make_perm_scratch_bytes(int m) {
    int L = next_pow2(std::max(m, 1));
    return L <= kPermSmemMax ? 0 : (size_t)L * (sizeof(uint64_t) + sizeof(int));
}

void launch_make_perm(unsigned long long seed, long long epoch, int m, int *perm,
                      uint64_t *keybuf, int *idxbuf, cudaStream_t st) {
    int L = next_pow2(std::max(m, 1));
    if (L <= kPermSmemMax) {
        size_t sm = (size_t)L * (sizeof(uint64_t) + sizeof(int));
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_perm_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kPermSmemMax * (int)(sizeof(uint64_t) + sizeof(int)));
            attr_set = true;
        }
        k_perm_smem<<<1, 1024, sm, st>>>(seed, epoch, m, L, perm);
        return;
    }
    int nb = ceil_div(L, 256);
    k_perm_fill<<<nb, 256, 0, st>>>(seed, epoch, m, L, keybuf, idxbuf);
    for (int k = 2; k <= L; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) k_perm_step<<<nb, 256, 0, st>>>(L, j, k, keybuf, idxbuf);
    k_perm_copy<<<ceil_div(m, 256), 256, 0, st>>>(m, idxbuf, perm);
}

// ---------------------------------------------------------------------------
// Plain cost materialisation for general d (CUDA cores, 16 x 16 tiles).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_cost_plain(int m, int n, int d, const Real *__restrict__ X,
                             const Real *__restrict__ Y, Real *__restrict__ C, bool euclid) {
    __shared__ Real xs[16][17], ys[16][17];
    int ti = threadIdx.y, tj = threadIdx.x;
    int i = blockIdx.y * 16 + ti, j = blockIdx.x * 16 + tj;
    Real acc = 0;
    for (int k0 = 0; k0 < d; k0 += 16) {
        int kk = k0 + tj;
        xs[ti][tj] = (i < m && kk < d) ? X[(size_t)i * d + kk] : Real(0);
        int jj = blockIdx.x * 16 + ti;
        ys[ti][tj] = (jj < n && kk < d) ? Y[(size_t)jj * d + kk] : Real(0);
        __syncthreads();
        int kmax = min(16, d - k0);
        for (int k = 0; k < kmax; ++k) {
            // ascending k, every operation rounded on its own (no contraction)
            if constexpr (std::is_same<Real, double>::value) {
                const double dl = dsub(xs[ti][k], ys[tj][k]);
                acc = dadd(acc, dmul(dl, dl));
            } else {
                const float dl = __fsub_rn(xs[ti][k], ys[tj][k]);
                acc = __fadd_rn(acc, __fmul_rn(dl, dl));
            }
        }
        __syncthreads();
    }
    if (i < m && j < n) C[(size_t)i * n + j] = euclid ? sqrt(acc) : acc;
}

template <typename Real>
void launch_cost_plain(int m, int n, int d, const Real *X, const Real *Y, Real *C, cudaStream_t st,
                       bool euclid) {
    dim3 blk(16, 16), grd(ceil_div(n, 16), ceil_div(m, 16));
    k_cost_plain<Real><<<grd, blk, 0, st>>>(m, n, d, X, Y, C, euclid);
}

template void launch_cost_plain<float>(int, int, int, const float *, const float *, float *, cudaStream_t, bool);
template void launch_cost_plain<double>(int, int, int, const double *, const double *, double *, cudaStream_t,
                                        bool);

}  // namespace srot
