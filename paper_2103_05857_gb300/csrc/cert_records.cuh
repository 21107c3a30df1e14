// cert_records.cuh -- the certificate of Thm 2 for one instance, taken by
// one CTA from the plan's atom records (its nonzeros with double-float
// weights), for the batched speculative form (FP32 plans, points with d = 3).
//
//   s_j = sum_i t_ij exactly (64-bit fixed point: integer additions do not
//         depend on the order in which threads add), q_j = rho (s_j - b_j);
//   f = <C, T> + ||q||^2 / (2 rho);
//   g = sum_i ( <t_i, c_i + q> - a_i min_j (c_ij + q_j) ),
// the LMO vertex of each row taken over all columns with FP32 keys of
// c_ij + q_j (ties to the smallest j) and evaluated in FP64.
#pragma once

#include "atoms.cuh"
#include "common.cuh"

namespace srot {

__device__ inline float rec_cost3(float x0, float x1, float x2, float4 y) {
    const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
    return fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0)));
}

// Fixed-point scale for exact column sums: every column sum is at most the
// plan's total mass sum_i a_i < 2^e2, so sums of 2^(61 - e2)-scaled weights
// fit a signed 64-bit integer.
__device__ inline int rec_fixed_exp(double total_mass) {
    int e2 = 0;
    frexp(total_mass > 1.0 ? total_mass : 1.0, &e2);
    return 61 - e2;
}

// sum_i a_i in a fixed order (per-thread strides, warp trees, warps in
// order); red: one double per warp. All threads of the CTA.
__device__ inline double rec_total_mass(const float *a, int m, double *red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x / kWarp;
    double s = 0.0;
    for (int i = tid; i < m; i += blockDim.x) s += (double)a[i];
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Column sums from the records into csum (n words), then q_j = rho (s_j -
// b_j) in place as doubles. All threads of the CTA.
__device__ inline void rec_records_to_q(const int4 *grec, int m, int n, const float *b, double rho, int fx,
                                        unsigned long long *csum) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = tid; j < n; j += nt) csum[j] = 0ull;
    __syncthreads();
    for (int i = tid; i < m; i += nt) {  // one row per thread: many records in flight
        const int4 *g = grec + (size_t)i * kAtomRecord;
        const int c = g[0].x;
        for (int k = 0; k < c; ++k) {
            const int4 at = g[1 + k];
            const double t = (double)__int_as_float(at.y) + (double)__int_as_float(at.z);
            if (t > 0.0) atomicAdd(&csum[at.x], (unsigned long long)__double2ll_rn(ldexp(t, fx)));
        }
    }
    __syncthreads();
    double *q = reinterpret_cast<double *>(csum);
    for (int j = tid; j < n; j += nt) {
        const double sj = ldexp((double)(long long)csum[j], -fx);
        q[j] = rho * (sj - (double)b[j]);
    }
    __syncthreads();
}

struct RecCert {
    double f, g, feas;
};

// The certificate of one instance by the whole CTA. csum: n words of
// scratch, holding q_j (doubles) on return; qf: n floats of scratch (the
// FP32 rounding of q for the LMO keys); jrow: kRecRowChunk ints of scratch;
// ys: the target points; red: 6 doubles per warp. Every thread returns the
// same values. GB300 issues an FP64 warp instruction at a small fraction of
// the FP32 rate whatever the number of active lanes, so the FP64 work runs
// one row per thread (32 rows per instruction): first the LMO vertex of
// each row (one warp per row, FP32 keys only), then per thread its row's
// sums over the atoms.
constexpr int kRecRowChunk = 4096;

__device__ inline RecCert rec_certificate(const int4 *grec, int m, int n, const float *X, const float4 *ys,
                                          const float *a, const float *b, double rho, int fx,
                                          unsigned long long *csum, float *qf, int *jrow, double *red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x / kWarp;
    const unsigned FULL = 0xffffffffu;
    rec_records_to_q(grec, m, n, b, rho, fx, csum);
    const double *q = reinterpret_cast<const double *>(csum);
    for (int j = tid; j < n; j += blockDim.x) qf[j] = (float)q[j];
    __syncthreads();
    double lin = 0.0, tq = 0.0, amin = 0.0;
    float feas = 0.f;
    for (int r0 = 0; r0 < m; r0 += kRecRowChunk) {
        const int r1 = min(m, r0 + kRecRowChunk);
        // (a) LMO vertex of each row, c_ij + q_j in FP32 (the operations of
        // rec_cost3, on row pairs in packed FP32x2), ties to the smallest j;
        // four rows per warp pass, so each (y_j, q_j) read from shared
        // memory serves four rows
        for (int i0 = r0 + 4 * warp; i0 < r1; i0 += 4 * nw) {
            float2 x0[2], x1[2], x2[2];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int ra = min(i0 + 2 * p, r1 - 1), rb = min(i0 + 2 * p + 1, r1 - 1);
                x0[p] = make_float2(X[(size_t)ra * 3], X[(size_t)rb * 3]);
                x1[p] = make_float2(X[(size_t)ra * 3 + 1], X[(size_t)rb * 3 + 1]);
                x2[p] = make_float2(X[(size_t)ra * 3 + 2], X[(size_t)rb * 3 + 2]);
            }
            float best[4];
            int bj[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                best[r] = __int_as_float(0x7f800000);  // +inf; a column index in range even if no
                bj[r] = min(lane, n - 1);               // value is below it
            }
            for (int j = lane; j < n; j += kWarp) {
                const float4 y = ys[j];
                const float qj = qf[j];
                const float2 ny0 = make_float2(-y.x, -y.x), ny1 = make_float2(-y.y, -y.y),
                             ny2 = make_float2(-y.z, -y.z), q2 = make_float2(qj, qj);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float2 d0 = __fadd2_rn(x0[p], ny0), d1 = __fadd2_rn(x1[p], ny1),
                                 d2 = __fadd2_rn(x2[p], ny2);
                    float2 c = __fmul2_rn(d0, d0);
                    c = __ffma2_rn(d1, d1, c);
                    c = __ffma2_rn(d2, d2, c);
                    c = __fadd2_rn(c, q2);
                    if (c.x < best[2 * p]) { best[2 * p] = c.x; bj[2 * p] = j; }
                    if (c.y < best[2 * p + 1]) { best[2 * p + 1] = c.y; bj[2 * p + 1] = j; }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t kb = f2key(best[r]);
                const uint32_t wk = __reduce_min_sync(FULL, kb);
                const int jm = __reduce_min_sync(FULL, kb == wk ? bj[r] : 0x7FFFFFFF);
                if (lane == 0 && i0 + r < r1) jrow[i0 + r - r0] = jm;
            }
        }
        __syncthreads();
        // (b) one row per thread, FP64: <t_i, c_i>, <t_i, q>, a_i (c_ij* + q_j*)
        for (int i = r0 + tid; i < r1; i += blockDim.x) {
            const float x0 = X[(size_t)i * 3], x1 = X[(size_t)i * 3 + 1], x2 = X[(size_t)i * 3 + 2];
            const int4 *g = grec + (size_t)i * kAtomRecord;
            const int c = g[0].x;
            double l1 = 0.0, l2 = 0.0, l3 = 0.0;
            for (int k = 0; k < c; ++k) {
                const int4 at = g[1 + k];
                const double t = (double)__int_as_float(at.y) + (double)__int_as_float(at.z);
                l1 += t * (double)rec_cost3(x0, x1, x2, ys[at.x]);
                l2 += t * q[at.x];
                l3 += t;
            }
            const int jm = min(max(jrow[i - r0], 0), n - 1);
            const double ai = (double)a[i];
            lin += l1;
            tq += l2;
            amin += ai * ((double)rec_cost3(x0, x1, x2, ys[jm]) + q[jm]);
            const float fa = (float)ai;
            feas = fmaxf(feas, fabsf((float)(l3 - ai)) / (fa > 0.f ? fa : 1e-30f));
        }
        __syncthreads();  // jrow is refilled by the next chunk
    }
    double rr = 0.0;  // ||q||^2
    for (int j = tid; j < n; j += blockDim.x) rr += q[j] * q[j];
    lin = warp_sum(lin);
    tq = warp_sum(tq);
    amin = warp_sum(amin);
    rr = warp_sum(rr);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) feas = fmaxf(feas, __shfl_xor_sync(FULL, feas, o));
    if (lane == 0) {
        red[6 * warp] = lin;
        red[6 * warp + 1] = tq;
        red[6 * warp + 2] = amin;
        red[6 * warp + 3] = (double)feas;
        red[6 * warp + 4] = rr;
    }
    __syncthreads();
    double L = 0.0, Q = 0.0, A2 = 0.0, FE = 0.0, R2 = 0.0;
    for (int w = 0; w < nw; ++w) {
        L += red[6 * w];
        Q += red[6 * w + 1];
        A2 += red[6 * w + 2];
        FE = fmax(FE, red[6 * w + 3]);
        R2 += red[6 * w + 4];
    }
    __syncthreads();
    RecCert cert;
    cert.f = L + (rho > 0.0 ? 0.5 * R2 / rho : 0.0);
    cert.g = (L + Q) - A2;
    cert.feas = FE;
    return cert;
}

}  // namespace srot
