// metrics.cu -- the evaluation metrics (v) and (vi) of Sec. 5 against a
// reference plan T_lp (the paper's T*_LP, the optimal plan of the unrelaxed
// transport problem):
//   e_m = ||T - T_lp|| / ||T_lp||                (Frobenius norm)
//   e_v = |<T, C> - <T_lp, C>| / |<T_lp, C>|
// One pass over T and T_lp (and C when it is given; d = 3 points evaluate the
// cost on the fly exactly as the solver does), HBM-bound: 2 m n (or 3 m n)
// elements read once. Each warp takes whole rows. FP64 plans are summed in
// FP64; FP32 plans form their products in FP32 and sum them per lane with
// Kahan compensation (GB300's FP64 pipe, 1/64 of the FP32 rate, would make
// an FP64 sum of every entry the bottleneck), then in FP64 across lanes. The
// order is fixed (lane strides, a fixed shuffle tree, warps in order, blocks
// in order), so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "step.cuh"

namespace srot {

namespace {

constexpr int kMetThreads = 256;
constexpr int kMetWarps = kMetThreads / kWarp;
constexpr int kMetMaxBlocks = 152 * 8;

template <typename Real>
__device__ inline Real met_cost(const LpMetricsArgs<Real> &A, int i, int j) {
    if (A.C) return A.C[(size_t)i * A.n + j];
    const Real *x = A.X + (size_t)i * 3;
    const Real *y = A.Y + (size_t)j * 3;
    if constexpr (std::is_same<Real, float>::value) {
        const float d0 = __fsub_rn(x[0], y[0]), d1 = __fsub_rn(x[1], y[1]), d2 = __fsub_rn(x[2], y[2]);
        if (A.euclid)  // the materialised Euclidean cost: ascending sum, no contraction, then sqrt
            return sqrtf(__fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2)));
        return fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0)));  // the solver's on-the-fly form
    } else {
        const double d0 = dsub(x[0], y[0]), d1 = dsub(x[1], y[1]), d2 = dsub(x[2], y[2]);
        const double s = dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2));
        return A.euclid ? sqrt(s) : s;
    }
}

__device__ inline double met_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// part[4 b + k], k: 0 = sum (t - l)^2, 1 = sum l^2, 2 = sum t c, 3 = sum l c
template <typename Real>
__global__ void __launch_bounds__(kMetThreads) k_lp_metrics(LpMetricsArgs<Real> A, double *part) {
    __shared__ double acc[kMetWarps][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if constexpr (std::is_same<Real, float>::value) {
        float h[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
        auto kahan = [&](int k, float x) {
            const float y = __fsub_rn(x, c[k]);
            const float tt = __fadd_rn(h[k], y);
            c[k] = __fsub_rn(__fsub_rn(tt, h[k]), y);
            h[k] = tt;
        };
        for (long long i = (long long)blockIdx.x * kMetWarps + warp; i < A.m; i += (long long)gridDim.x * kMetWarps) {
            const float *t = A.T + (size_t)i * A.n;
            const float *l = A.L + (size_t)i * A.n;
            for (int j = lane; j < A.n; j += kWarp) {
                const float tv = t[j], lv = l[j], cv = met_cost(A, (int)i, j);
                const float dd = __fsub_rn(tv, lv);
                kahan(0, __fmul_rn(dd, dd));
                kahan(1, __fmul_rn(lv, lv));
                kahan(2, __fmul_rn(tv, cv));
                kahan(3, __fmul_rn(lv, cv));
            }
        }
        s0 = (double)h[0] - (double)c[0];
        s1 = (double)h[1] - (double)c[1];
        s2 = (double)h[2] - (double)c[2];
        s3 = (double)h[3] - (double)c[3];
    } else {
        for (long long i = (long long)blockIdx.x * kMetWarps + warp; i < A.m; i += (long long)gridDim.x * kMetWarps) {
            const double *t = A.T + (size_t)i * A.n;
            const double *l = A.L + (size_t)i * A.n;
            for (int j = lane; j < A.n; j += kWarp) {
                const double tv = t[j], lv = l[j], cv = met_cost(A, (int)i, j);
                const double dd = tv - lv;
                s0 += dd * dd;
                s1 += lv * lv;
                s2 += tv * cv;
                s3 += lv * cv;
            }
        }
    }
    s0 = met_warp_sum(s0);
    s1 = met_warp_sum(s1);
    s2 = met_warp_sum(s2);
    s3 = met_warp_sum(s3);
    if (lane == 0) {
        acc[warp][0] = s0;
        acc[warp][1] = s1;
        acc[warp][2] = s2;
        acc[warp][3] = s3;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < kMetWarps; ++w) v += acc[w][threadIdx.x];
        part[4 * blockIdx.x + threadIdx.x] = v;
    }
}

// out[0..3]: the four sums over every block, in block order
__global__ void k_lp_metrics_final(const double *part, int nblocks, double *out) {
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += part[4 * b + threadIdx.x];
        out[threadIdx.x] = v;
    }
}

}  // namespace

int lp_metrics_blocks(int m) {
    int b = (m + kMetWarps - 1) / kMetWarps;
    return b < 1 ? 1 : (b > kMetMaxBlocks ? kMetMaxBlocks : b);
}

template <typename Real>
void launch_lp_metrics(const LpMetricsArgs<Real> &A, double *part, double *out, cudaStream_t st) {
    const int nb = lp_metrics_blocks(A.m);
    k_lp_metrics<Real><<<nb, kMetThreads, 0, st>>>(A, part);
    k_lp_metrics_final<<<1, 32, 0, st>>>(part, nb, out);
}

template void launch_lp_metrics<float>(const LpMetricsArgs<float> &, double *, double *, cudaStream_t);
template void launch_lp_metrics<double>(const LpMetricsArgs<double> &, double *, double *, cudaStream_t);

}  // namespace srot
