// solve_fw.cu -- one step of full (not block-coordinate) Frank-Wolfe, Alg. A.1.
//
// Every row's LMO vertex j*_i is taken at the same plan T (the certificate's
// row pass writes them), S = (a_i e_{j*_i}) is the vertex of the product of
// simplices, d = S - T, and the step is
//   decay:        gamma = 2 / (it + 2),
//   line search:  gamma = clip(g / (rho ||(T - S)^T 1||^2), 0, 1)
// where g = <T - S, grad f(T)> is the gap of the certificate (Thm 2) and
// (T - S)^T 1 = s - sum_i a_i e_{j*_i} is the only part of d the quadratic
// penalty sees. Then T <- (1 - gamma) T + gamma S in one pass over T.
//
// The column sums of S are taken per column in ascending row order (rows are
// staged through shared memory in chunks), so the line search is the same
// from run to run.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "step.cuh"

namespace srot {

namespace {

constexpr int kFwThreads = 256;
constexpr int kFwChunk = 2048;

// Partial sums of u_j^2, u = s - S^T 1, one per block of 256 columns.
template <typename Real>
__global__ void __launch_bounds__(kFwThreads)
k_fw_usq(int m, int n, const int *__restrict__ js, const Real *__restrict__ a, const Real *__restrict__ b,
         const double *__restrict__ r64, double *__restrict__ upart) {
    __shared__ int sj[kFwChunk];
    __shared__ double sa[kFwChunk];
    __shared__ double red[kFwThreads / kWarp];
    const int j = blockIdx.x * kFwThreads + threadIdx.x;
    double acc = 0.0;
    for (int i0 = 0; i0 < m; i0 += kFwChunk) {
        const int len = min(kFwChunk, m - i0);
        __syncthreads();
        for (int t = threadIdx.x; t < len; t += kFwThreads) {
            sj[t] = js[i0 + t];
            sa[t] = (double)a[i0 + t];
        }
        __syncthreads();
        for (int t = 0; t < len; ++t)
            if (sj[t] == j) acc += sa[t];
    }
    double u2 = 0.0;
    if (j < n) {
        const double s = r64[j] + (double)b[j];  // r64 = s - b
        const double u = s - acc;
        u2 = u * u;
    }
    u2 = warp_sum(u2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = u2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kFwThreads / kWarp; ++w) t += red[w];
        upart[blockIdx.x] = t;
    }
}

__global__ void k_fw_gamma(const double *__restrict__ upart, int nparts, const double *__restrict__ cert,
                           double rho, double *__restrict__ gamma) {
    if (threadIdx.x != 0) return;
    double uu = 0.0;
    for (int k = 0; k < nparts; ++k) uu += upart[k];
    *gamma = line_search<double>(cert[kCertG], uu, rho, 1.0);
}

__global__ void k_fw_set_gamma(double g, double *__restrict__ gamma) {
    if (threadIdx.x == 0) *gamma = g;
}

// T <- (1 - gamma) T + gamma a_i e_{j*_i}; one block per row at a time.
template <typename Real>
__global__ void k_fw_update(int m, int n, Real *__restrict__ T, const int *__restrict__ js,
                            const Real *__restrict__ a, const double *__restrict__ gamma) {
    const double gam = *gamma;
    for (int i = blockIdx.x; i < m; i += gridDim.x) {
        Real *ti = T + (size_t)i * n;
        const int jstar = js[i];
        if constexpr (std::is_same<Real, double>::value) {
            const double omg = dsub(1.0, gam), ga = dmul(gam, a[i]);
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                double t = dmul(omg, ti[j]);
                if (j == jstar) t = dadd(t, ga);
                ti[j] = t;
            }
        } else {
            const float gf = (float)gam, omg = 1.f - gf, ga = gf * a[i];
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                float t = omg * ti[j];
                if (j == jstar) t = t + ga;
                ti[j] = t;
            }
        }
    }
}

}  // namespace

int fw_upart_size(int n) { return ceil_div(n, kFwThreads); }

template <typename Real>
void launch_fw_step(const Inst<Real> &in, Real *T, const int *js, const double *r64,
                    const double *cert, int step, long long it, double rho, double *upart,
                    double *gamma_dev, cudaStream_t st) {
    const int m = in.m, n = in.n;
    if (step == SR_OT_ELS) {
        const int nb = fw_upart_size(n);
        k_fw_usq<Real><<<nb, kFwThreads, 0, st>>>(m, n, js, in.a, in.b, r64, upart);
        k_fw_gamma<<<1, 32, 0, st>>>(upart, nb, cert, rho, gamma_dev);
    } else {
        k_fw_set_gamma<<<1, 32, 0, st>>>(2.0 / ((double)it + 2.0), gamma_dev);
    }
    const int blocks = std::min(m, 152 * 8);
    k_fw_update<Real><<<blocks, 256, 0, st>>>(m, n, T, js, in.a, gamma_dev);
}

template void launch_fw_step<float>(const Inst<float> &, float *, const int *, const double *,
                                    const double *, int, long long, double, double *, double *,
                                    cudaStream_t);
template void launch_fw_step<double>(const Inst<double> &, double *, const int *, const double *,
                                     const double *, int, long long, double, double *, double *,
                                     cudaStream_t);

}  // namespace srot
