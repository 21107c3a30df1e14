// adjoint.cu -- gradients of the optimal value through the envelope theorem.
//
// At an optimal plan T of min_T <C, T> + (rho/2) ||T^T 1 - b||^2 over the
// product of simplices {T >= 0, T 1 = a} (Sec. 2, the semi-relaxed problem in
// this library's row orientation), the derivative of the optimal value with
// respect to the data is the partial derivative of the objective at fixed T:
//   dC = T,
//   dX = 2 (diag(T 1) X - T Y),      (C_ij = ||x_i - y_j||^2)
//   dY = 2 (diag(T^T 1) Y - T^T X),
//   db = -rho (T^T 1 - b).
// The paper does not differentiate its solver; this is the library's backward
// pass.
//
// One pass reads T once. A CTA of 256 threads owns a tile of `rh` rows x 256
// columns (one column per thread). Per row it accumulates the column partials
// t_ij (x_i, 1) in registers and forms the row partials t_ij (y_j, 1), which a
// warp reduce-scatter (31 shuffles for 32 values) folds across the warp's 32
// columns for R = 32 / P rows at a time, P = the padded width d + 1. The
// per-warp row partials are summed in a fixed order in shared memory; column
// partials (per row band) and row partials (per column tile) go to a
// workspace, and two small kernels reduce them in FP64 in a fixed order, so
// the result does not depend on scheduling.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace srot {

namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjWarps = kAdjThreads / kWarp;

// rows staged per chunk: the per-warp row-partial buffer stays <= 32 KiB
template <typename Real, int P>
constexpr int adj_chunk() {
    return (32768 / (kAdjWarps * P * (int)sizeof(Real))) < 64 ? (32768 / (kAdjWarps * P * (int)sizeof(Real)))
                                                              : 64;
}

// Index of the last instance whose `key` prefix is <= x (instances sorted by key).
template <typename F>
__device__ inline int find_inst(int ninst, long long x, F key) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (key(mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// After the call, lane l holds the warp-wide sum of v[l] (all 32 lanes'
// values at index l): a butterfly that halves the live values per step.
template <typename Real>
__device__ inline Real reduce_scatter32(Real (&v)[32], int lane) {
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const Real send = upper ? v[q] : v[q + half];
            const Real keep = upper ? v[q + half] : v[q];
            v[q] = keep + __shfl_xor_sync(FULL, send, half);
        }
    }
    return v[0];
}

template <typename Real, int P>
__global__ void __launch_bounds__(kAdjThreads) k_adj_tiles(AdjArgs<Real> A) {
    constexpr int R = 32 / P;
    constexpr int CH = adj_chunk<Real, P>();
    __shared__ __align__(16) Real xs[CH][P];
    __shared__ __align__(16) Real rsm[CH][kAdjWarps][P];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = find_inst(A.ninst, (long long)blockIdx.x, [&](int q) { return (long long)A.inst[q].tile0; });
    const AdjInst I = A.inst[k];
    const int t = (int)blockIdx.x - I.tile0;
    const int band = t / I.ncol, ct = t - band * I.ncol;
    const int i0 = band * I.rh, i1 = min(I.m, i0 + I.rh);
    const int j = ct * kAdjThreads + tid;
    const bool jv = j < I.n;
    const int d = A.d;
    const Real *Tm = A.T + I.oT;
    Real *dCm = A.dC ? A.dC + I.oT : nullptr;

    Real y[P], cacc[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
        y[c] = (c < d && jv && A.Y) ? A.Y[I.oY + (size_t)j * d + c] : (c == d ? Real(1) : Real(0));
        cacc[c] = Real(0);
    }
    const bool want_x = A.X != nullptr;

    for (int c0 = i0; c0 < i1; c0 += CH) {
        const int rows = min(CH, i1 - c0);
        __syncthreads();  // the previous chunk's buffers are consumed
        for (int e = tid; e < CH * P; e += kAdjThreads) {
            const int r = e / P, c = e - r * P;
            Real v = Real(0);
            if (r < rows) v = c < d ? (want_x ? A.X[I.oX + (size_t)(c0 + r) * d + c] : Real(0))
                                    : (c == d ? Real(1) : Real(0));
            xs[r][c] = v;
        }
        __syncthreads();
        for (int g = 0; g < rows; g += R) {
            Real tv[R];
#pragma unroll
            for (int r = 0; r < R; ++r)
                tv[r] = (jv && g + r < rows) ? Tm[(size_t)(c0 + g + r) * I.n + j] : Real(0);
            Real v[32];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (dCm && jv && g + r < rows) dCm[(size_t)(c0 + g + r) * I.n + j] = tv[r];
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    cacc[c] += tv[r] * xs[g + r][c];
                    v[r * P + c] = tv[r] * y[c];
                }
            }
            const Real s = reduce_scatter32(v, lane);
            const int r = lane / P, c = lane - (lane / P) * P;
            if (g + r < rows) rsm[g + r][warp][c] = s;
        }
        __syncthreads();
        for (int e = tid; e < rows * P; e += kAdjThreads) {
            const int r = e / P, c = e - r * P;
            Real s = Real(0);
#pragma unroll
            for (int w = 0; w < kAdjWarps; ++w) s += rsm[r][w][c];
            A.rowpart[I.orp + ((size_t)ct * I.m + (c0 + r)) * P + c] = s;
        }
    }
    if (jv) {
#pragma unroll
        for (int c = 0; c < P; ++c) A.colpart[I.ocp + ((size_t)band * I.n + j) * P + c] = cacc[c];
    }
}

// dY and db from the column partials (sum over row bands, ascending).
template <typename Real, int P>
__global__ void k_adj_cols(AdjArgs<Real> A) {
    const int d = A.d;
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < A.total_cols;
         gi += (long long)gridDim.x * blockDim.x) {
        const int k = find_inst(A.ninst, gi, [&](int q) { return A.inst[q].col0; });
        const AdjInst I = A.inst[k];
        const int j = (int)(gi - I.col0);
        double acc[P];
#pragma unroll
        for (int c = 0; c < P; ++c) acc[c] = 0.0;
        for (int band = 0; band < I.nbands; ++band) {
            const Real *p = A.colpart + I.ocp + ((size_t)band * I.n + j) * P;
#pragma unroll
            for (int c = 0; c < P; ++c) acc[c] += (double)p[c];
        }
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < P; ++c)
            if (c == d) s = acc[c];
        if (A.dY) {
#pragma unroll
            for (int c = 0; c < P; ++c)
                if (c < d) {
                    const double yv = (double)A.Y[I.oY + (size_t)j * d + c];
                    A.dY[I.oY + (size_t)j * d + c] = (Real)(2.0 * (s * yv - acc[c]));
                }
        }
        if (A.db) A.db[I.ob + j] = (Real)(-A.rho * (s - (double)A.b[I.ob + j]));
    }
}

// dX from the row partials (sum over column tiles, ascending).
template <typename Real, int P>
__global__ void k_adj_rows(AdjArgs<Real> A) {
    const int d = A.d;
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < A.total_rows;
         gi += (long long)gridDim.x * blockDim.x) {
        const int k = find_inst(A.ninst, gi, [&](int q) { return A.inst[q].row0; });
        const AdjInst I = A.inst[k];
        const int i = (int)(gi - I.row0);
        double acc[P];
#pragma unroll
        for (int c = 0; c < P; ++c) acc[c] = 0.0;
        for (int ct = 0; ct < I.ncol; ++ct) {
            const Real *p = A.rowpart + I.orp + ((size_t)ct * I.m + i) * P;
#pragma unroll
            for (int c = 0; c < P; ++c) acc[c] += (double)p[c];
        }
        double rs = 0.0;
#pragma unroll
        for (int c = 0; c < P; ++c)
            if (c == d) rs = acc[c];
#pragma unroll
        for (int c = 0; c < P; ++c)
            if (c < d) {
                const double xv = (double)A.X[I.oX + (size_t)i * d + c];
                A.dX[I.oX + (size_t)i * d + c] = (Real)(2.0 * (rs * xv - acc[c]));
            }
    }
}

template <typename Real, int P>
void launch_p(const AdjArgs<Real> &A, cudaStream_t st) {
    k_adj_tiles<Real, P><<<A.total_tiles, kAdjThreads, 0, st>>>(A);
    if (A.dY || A.db) {
        const int blocks = (int)std::min<long long>((A.total_cols + 255) / 256, 152 * 8);
        k_adj_cols<Real, P><<<std::max(blocks, 1), 256, 0, st>>>(A);
    }
    if (A.dX) {
        const int blocks = (int)std::min<long long>((A.total_rows + 255) / 256, 152 * 8);
        k_adj_rows<Real, P><<<std::max(blocks, 1), 256, 0, st>>>(A);
    }
}

}  // namespace

int adj_width(int d) {
    int p = 4;
    while (p < d + 1) p <<= 1;
    return p;
}

AdjTotals adj_plan(int ninst, const int *m, const int *n, int d, AdjInst *out) {
    const int P = adj_width(d);
    long long ncol_total = 0;
    for (int k = 0; k < ninst; ++k) ncol_total += (n[k] + kAdjThreads - 1) / kAdjThreads;
    // enough tiles to fill the GPU (152 SMs x 8 CTAs), rows per band a multiple of 64
    const long long target = 152 * 8;
    const long long f = std::max<long long>(1, (target + ncol_total - 1) / std::max<long long>(ncol_total, 1));
    AdjTotals tot{0, 0, 0, 0, 0};
    for (int k = 0; k < ninst; ++k) {
        AdjInst &I = out[k];
        I.m = m[k];
        I.n = n[k];
        I.ncol = (n[k] + kAdjThreads - 1) / kAdjThreads;
        const long long maxb = (m[k] + 63) / 64;
        const int nb0 = (int)std::min<long long>(f, maxb);
        int rh = (m[k] + nb0 - 1) / nb0;
        rh = ((rh + 63) / 64) * 64;
        I.rh = rh;
        I.nbands = (m[k] + rh - 1) / rh;
        I.tile0 = (int)tot.tiles;
        I.col0 = tot.cols;
        I.row0 = tot.rows;
        I.ocp = tot.colpart;
        I.orp = tot.rowpart;
        tot.tiles += (long long)I.nbands * I.ncol;
        tot.cols += n[k];
        tot.rows += m[k];
        tot.colpart += (long long)I.nbands * n[k] * P;
        tot.rowpart += (long long)I.ncol * m[k] * P;
    }
    return tot;
}

template <typename Real>
bool launch_adjoint(const AdjArgs<Real> &A, cudaStream_t st) {
    switch (adj_width(A.d)) {
        case 4: launch_p<Real, 4>(A, st); return true;
        case 8: launch_p<Real, 8>(A, st); return true;
        case 16: launch_p<Real, 16>(A, st); return true;
        case 32: launch_p<Real, 32>(A, st); return true;
        default: return false;
    }
}

template bool launch_adjoint<float>(const AdjArgs<float> &, cudaStream_t);
template bool launch_adjoint<double>(const AdjArgs<double> &, cudaStream_t);

}  // namespace srot
