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
// One pass reads T once. A CTA of 8 warps owns a tile of `rh` rows x TW
// columns, TW = 32 lanes x CPT columns per lane (16 bytes of T per lane per
// row: 4 FP32 or 2 FP64 columns; one column when d + 1 > 8). Each warp takes
// its own groups of R = 32 / P rows (P = the padded width of d + 1) over all
// TW columns: per row it accumulates the column partials t_ij (x_i, 1) in
// registers and the row partials sum_j t_ij (y_j, 1), which a warp
// reduce-scatter (31 shuffles for 32 values) completes for the tile, so row
// partials go straight to a workspace with no block barrier in the loop.
// The 8 warps' column partials are summed in a fixed order at the end. A
// small finishing kernel reduces the per-band and per-tile partials in FP64
// in a fixed order, so the result does not depend on scheduling.
//
// The same pass gives the colour-transfer tail (Sec. 5.1 and the metrics
// (iii), (iv) of Sec. 5): the row partials sum_j T_ij (y_j, 1) are the
// numerator and denominator of the barycentric projection, the row and
// column sums the marginal errors, and the tiles count the zero entries.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace srot {

namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjWarps = kAdjThreads / kWarp;
constexpr int kFinThreads = 256;
constexpr int kAdjBandMax = 1024;  // rows of a band (adj_plan keeps rh <= this for the FP32 d <= 3 path)

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

// Columns per thread: 16 bytes of T per row while the per-column registers
// (2 CPT P) stay small, else one.
template <typename Real, int P>
constexpr int adj_cpt() { return P <= 8 ? 16 / (int)sizeof(Real) : 1; }

template <typename Real>
struct Vec16;
template <>
struct Vec16<float> { using T = float4; };
template <>
struct Vec16<double> { using T = double2; };

template <typename Real, int P>
__global__ void __launch_bounds__(kAdjThreads) k_adj_tiles(AdjArgs<Real> A) {
    constexpr int R = 32 / P;
    constexpr int CPT = adj_cpt<Real, P>();
    constexpr int TW = kWarp * CPT;                   // columns of a tile (one per lane x CPT)
    constexpr bool V16 = CPT * sizeof(Real) == 16;
    constexpr int QC = (32768 / (kAdjWarps * TW * (int)sizeof(Real))) < P
                           ? (32768 / (kAdjWarps * TW * (int)sizeof(Real))) : P;  // components per pass
    __shared__ __align__(16) Real csm[kAdjWarps][QC][TW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = find_inst(A.ninst, (long long)blockIdx.x, [&](int q) { return (long long)A.inst[q].tile0; });
    const AdjInst I = A.inst[k];
    const int t = (int)blockIdx.x - I.tile0;
    const int band = t / I.ncol, ct = t - band * I.ncol;
    const int i0 = band * I.rh, i1 = min(I.m, i0 + I.rh);
    const int j0 = ct * TW + lane * CPT;  // this lane's first column
    const int d = A.d;
    const Real *Tm = A.T + I.oT;
    Real *dCm = A.dC ? A.dC + I.oT : nullptr;
    // 16-byte row accesses when every row starts on a 16-byte boundary
    const bool vec = V16 && (I.n % CPT == 0) && ((reinterpret_cast<uintptr_t>(Tm) & 15) == 0) &&
                     (!dCm || (reinterpret_cast<uintptr_t>(dCm) & 15) == 0);
    const Real *Xm = A.X ? A.X + I.oX : nullptr;
    unsigned nzero = 0;  // zero entries of T seen by this thread (transfer statistics)

    // column partials: sum over the 8 warps in a fixed order, QC components at a time
    auto column_partials = [&](Real (&cacc)[CPT][P]) {
#pragma unroll
        for (int q0 = 0; q0 < P; q0 += QC) {
            __syncthreads();
#pragma unroll
            for (int qq = 0; qq < QC; ++qq)
#pragma unroll
                for (int c = 0; c < CPT; ++c) csm[warp][qq][lane * CPT + c] = cacc[c][q0 + qq];
            __syncthreads();
            for (int e = tid; e < QC * TW; e += kAdjThreads) {
                const int qq = e / TW, col = e - qq * TW;
                const int j = ct * TW + col;
                Real sum = Real(0);
#pragma unroll
                for (int w = 0; w < kAdjWarps; ++w) sum += csm[w][qq][col];
                if (j < I.n) A.colpart[I.ocp + ((size_t)band * I.n + j) * P + q0 + qq] = sum;
            }
        }
    };
    if constexpr (std::is_same<Real, float>::value && P == 4 && CPT == 4) {
        // FP32, d <= 3: column pairs as packed FP32x2 (two columns per
        // instruction), the band's (x_i, 1) staged once in shared memory
        __shared__ float4 xs[kAdjBandMax];
        for (int i = i0 + tid; i < i1; i += kAdjThreads) {
            float e[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) e[q] = q < d ? (Xm ? Xm[(size_t)i * d + q] : 0.f) : (q == d ? 1.f : 0.f);
            xs[i - i0] = make_float4(e[0], e[1], e[2], e[3]);
        }
        __syncthreads();
        float2 y2[2][4], ca2[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float yy[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = j0 + 2 * h + e;
                    yy[e] = (q < d && j < I.n && A.Y) ? A.Y[I.oY + (size_t)j * d + q] : (q == d ? 1.f : 0.f);
                }
                y2[h][q] = make_float2(yy[0], yy[1]);
                ca2[h][q] = make_float2(0.f, 0.f);
            }
        for (int r0 = i0 + warp * R; r0 < i1; r0 += kAdjWarps * R) {
            float4 tv[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const size_t off = (size_t)(r0 + r) * I.n + j0;
                if (vec) {
                    tv[r] = (r0 + r < i1 && j0 < I.n) ? __ldg(reinterpret_cast<const float4 *>(Tm + off))
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    float e[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) e[c] = (r0 + r < i1 && j0 + c < I.n) ? __ldg(Tm + off + c) : 0.f;
                    tv[r] = make_float4(e[0], e[1], e[2], e[3]);
                }
            }
            if (dCm) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r0 + r >= i1) break;
                    const size_t off = (size_t)(r0 + r) * I.n + j0;
                    const float e[4] = {tv[r].x, tv[r].y, tv[r].z, tv[r].w};
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (j0 + c < I.n) dCm[off + c] = e[c];
                }
            }
            if (A.zeros) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r0 + r >= i1) break;
                    const float e[4] = {tv[r].x, tv[r].y, tv[r].z, tv[r].w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) nzero += (j0 + c < I.n && e[c] == 0.f) ? 1u : 0u;
                }
            }
            float v[32];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 ta = make_float2(tv[r].x, tv[r].y), tb = make_float2(tv[r].z, tv[r].w);
                const float4 x4 = r0 + r < i1 ? xs[r0 + r - i0] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float xq[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 x2 = make_float2(xq[q], xq[q]);
                    ca2[0][q] = __ffma2_rn(ta, x2, ca2[0][q]);
                    ca2[1][q] = __ffma2_rn(tb, x2, ca2[1][q]);
                    const float2 a2 = __ffma2_rn(tb, y2[1][q], __fmul2_rn(ta, y2[0][q]));
                    v[r * 4 + q] = a2.x + a2.y;
                }
            }
            const float sres = reduce_scatter32(v, lane);
            const int r = lane / P, q = lane - (lane / P) * P;
            if (r0 + r < i1) A.rowpart[I.orp + ((size_t)ct * I.m + (r0 + r)) * P + q] = sres;
        }
        Real cacc[CPT][P];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cacc[0][q] = ca2[0][q].x;
            cacc[1][q] = ca2[0][q].y;
            cacc[2][q] = ca2[1][q].x;
            cacc[3][q] = ca2[1][q].y;
        }
        column_partials(cacc);
    } else {
        Real y[CPT][P], cacc[CPT][P];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int j = j0 + c;
#pragma unroll
            for (int q = 0; q < P; ++q) {
                y[c][q] = (q < d && j < I.n && A.Y) ? A.Y[I.oY + (size_t)j * d + q] : (q == d ? Real(1) : Real(0));
                cacc[c][q] = Real(0);
            }
        }

        // Each warp takes groups of R rows (warp w: groups w, w + 8, ...) over all
        // TW columns of the tile, so a row's partial over the tile is complete
        // after the warp's reduce-scatter: no block barrier in this loop.
        for (int r0 = i0 + warp * R; r0 < i1; r0 += kAdjWarps * R) {
            // all R rows are loaded before anything is stored (dC may not be
            // proven distinct from T), so the loads are in flight together
            Real tv[R][CPT];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool rv = r0 + r < i1;
                const size_t off = (size_t)(r0 + r) * I.n + j0;
                if (V16 && vec) {
                    typename Vec16<Real>::T w;
                    if (rv && j0 < I.n) w = __ldg(reinterpret_cast<const typename Vec16<Real>::T *>(Tm + off));
                    else w = typename Vec16<Real>::T{};
                    const Real *pw = reinterpret_cast<const Real *>(&w);
#pragma unroll
                    for (int c = 0; c < CPT; ++c) tv[r][c] = pw[c];
                } else {
#pragma unroll
                    for (int c = 0; c < CPT; ++c) tv[r][c] = (rv && j0 + c < I.n) ? __ldg(Tm + off + c) : Real(0);
                }
            }
            if (dCm) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r0 + r >= i1) break;
                    const size_t off = (size_t)(r0 + r) * I.n + j0;
#pragma unroll
                    for (int c = 0; c < CPT; ++c)
                        if (j0 + c < I.n) dCm[off + c] = tv[r][c];
                }
            }
            if (A.zeros) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r0 + r >= i1) break;
#pragma unroll
                    for (int c = 0; c < CPT; ++c) nzero += (j0 + c < I.n && tv[r][c] == Real(0)) ? 1u : 0u;
                }
            }
            Real v[32];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool rv = r0 + r < i1;
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const Real xq = q < d ? ((Xm && rv) ? Xm[(size_t)(r0 + r) * d + q] : Real(0))
                                          : (q == d ? Real(1) : Real(0));
                    Real acc = Real(0);
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        cacc[c][q] += tv[r][c] * xq;
                        acc += tv[r][c] * y[c][q];
                    }
                    v[r * P + q] = acc;
                }
            }
            const Real sres = reduce_scatter32(v, lane);
            const int r = lane / P, q = lane - (lane / P) * P;
            if (r0 + r < i1) A.rowpart[I.orp + ((size_t)ct * I.m + (r0 + r)) * P + q] = sres;
        }

        column_partials(cacc);
    }
    if (A.zeros) {
        const unsigned wz = __reduce_add_sync(0xffffffffu, nzero);
        if (lane == 0 && wz) atomicAdd(A.zeros + k, (unsigned long long)wz);
    }
}

// acc[c] = sum of p[k * stride + c] over k = 0 .. count-1 in ascending k;
// the loads of up to kBatch partials are issued before any is added. FP32
// partials are summed with compensation (Kahan) in FP32 and handed over in
// double (GB300's FP64 rate is a small fraction of its FP32 rate; the
// compensated sum is accurate to about one FP32 rounding of the total).
template <typename Real, int P>
__device__ inline void sum_partials(const Real *p, size_t stride, int count, double (&acc)[P]) {
    constexpr int kBatch = P <= 4 ? 8 : (P <= 8 ? 4 : 1);
    constexpr bool kF32 = sizeof(Real) == 4;
    Kahan32 ks[kF32 ? P : 1];
    for (int k0 = 0; k0 < count; k0 += kBatch) {
        Real buf[kBatch][P];
#pragma unroll
        for (int b = 0; b < kBatch; ++b)
#pragma unroll
            for (int c = 0; c < P; ++c) buf[b][c] = k0 + b < count ? __ldg(p + (size_t)(k0 + b) * stride + c) : Real(0);
#pragma unroll
        for (int b = 0; b < kBatch; ++b)
            if (k0 + b < count) {
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    if constexpr (kF32) ks[c].add((float)buf[b][c]);
                    else acc[c] += (double)buf[b][c];
                }
            }
    }
    if constexpr (kF32) {
#pragma unroll
        for (int c = 0; c < P; ++c) acc[c] = ks[c].value();
    }
}

// Deterministic block sum (fixed butterfly per warp, warps in order); the
// result is valid in thread 0. Every thread of the block must call it.
__device__ inline double block_sum_fixed(double v) {
    __shared__ double sh[kFinThreads / kWarp];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kFinThreads / kWarp; ++w) t += sh[w];
    return t;
}

// Finishing pass: each instance owns ceil(m / 256) row blocks (dX and the
// barycentric projection from the row partials, summed over column tiles in
// ascending order) followed by ceil(n / 256) column blocks (dY, db from the
// column partials, summed over row bands in ascending order); a block never
// spans two instances. With tpart, each block also leaves the sum of its
// squared marginal errors (rows: (T1 - a)_i^2, columns: (T^T 1 - b)_j^2).
template <typename Real, int P>
__global__ void __launch_bounds__(kFinThreads) k_adj_finish(AdjArgs<Real> A) {
    __shared__ int sk;
    if (threadIdx.x == 0) sk = find_inst(A.ninst, (long long)blockIdx.x, [&](int q) { return (long long)A.inst[q].fin0; });
    __syncthreads();
    const AdjInst I = A.inst[sk];
    const int d = A.d;
    const int rblocks = (I.m + kFinThreads - 1) / kFinThreads;
    const int lb = (int)blockIdx.x - I.fin0;
    double acc[P];
#pragma unroll
    for (int c = 0; c < P; ++c) acc[c] = 0.0;
    double sq = 0.0;  // squared marginal error of this thread's row or column
    if (lb < rblocks) {
        const int i = lb * kFinThreads + (int)threadIdx.x;
        if (i < I.m && (A.dX || A.xhat || A.tpart)) {
            sum_partials<Real, P>(A.rowpart + I.orp + (size_t)i * P, (size_t)I.m * P, I.ncol, acc);
            double rs = 0.0;
#pragma unroll
            for (int c = 0; c < P; ++c)
                if (c == d) rs = acc[c];
            if (A.dX) {
#pragma unroll
                for (int c = 0; c < P; ++c)
                    if (c < d) {
                        const double xv = (double)A.X[I.oX + (size_t)i * d + c];
                        A.dX[I.oX + (size_t)i * d + c] = (Real)(2.0 * (rs * xv - acc[c]));
                    }
            }
            if (A.xhat) {
#pragma unroll
                for (int c = 0; c < P; ++c)
                    if (c < d) A.xhat[I.oX + (size_t)i * d + c] = rs > 0.0 ? (Real)(acc[c] / rs) : Real(0);
            }
            if (A.tpart) {
                const double e = rs - (double)A.a[I.oa + i];
                sq = e * e;
            }
        }
    } else {
        const int j = (lb - rblocks) * kFinThreads + (int)threadIdx.x;
        if (j < I.n && (A.dY || A.db || A.tpart)) {
            sum_partials<Real, P>(A.colpart + I.ocp + (size_t)j * P, (size_t)I.n * P, I.nbands, acc);
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
            if (A.tpart) {
                const double e = s - (double)A.b[I.ob + j];
                sq = e * e;
            }
        }
    }
    if (A.tpart) {
        const double t = block_sum_fixed(sq);
        if (threadIdx.x == 0) A.tpart[blockIdx.x] = t;
    }
}

// Transfer statistics per instance from the finishing blocks' sums (in
// ascending block order) and the zero count.
template <typename Real>
__global__ void k_transfer_stats(AdjArgs<Real> A) {
    for (int k = threadIdx.x; k < A.ninst; k += blockDim.x) {
        const AdjInst I = A.inst[k];
        const int rblocks = (I.m + kFinThreads - 1) / kFinThreads, cblocks = (I.n + kFinThreads - 1) / kFinThreads;
        double r2 = 0.0, c2 = 0.0;
        for (int q = 0; q < rblocks; ++q) r2 += A.tpart[I.fin0 + q];
        for (int q = 0; q < cblocks; ++q) c2 += A.tpart[I.fin0 + rblocks + q];
        const double re = sqrt(r2), ce = sqrt(c2);
        A.tstats[4 * k + 0] = re;
        A.tstats[4 * k + 1] = ce;
        A.tstats[4 * k + 2] = re + ce;
        A.tstats[4 * k + 3] = (double)A.zeros[k] / ((double)I.m * (double)I.n);
    }
}

template <typename Real, int P>
void launch_p(const AdjArgs<Real> &A, cudaStream_t st) {
    k_adj_tiles<Real, P><<<A.total_tiles, kAdjThreads, 0, st>>>(A);
    if (A.dX || A.dY || A.db || A.xhat || A.tpart) k_adj_finish<Real, P><<<A.total_fin, kFinThreads, 0, st>>>(A);
    if (A.tpart && A.tstats && A.zeros) k_transfer_stats<Real><<<1, 128, 0, st>>>(A);
}

}  // namespace

int adj_width(int d) {
    int p = 4;
    while (p < d + 1) p <<= 1;
    return p;
}

int adj_cols_per_thread(int d, int elem_bytes) { return adj_width(d) <= 8 ? 16 / elem_bytes : 1; }

AdjTotals adj_plan(int ninst, const int *m, const int *n, int d, int elem_bytes, AdjInst *out) {
    const int P = adj_width(d);
    const int TW = kWarp * adj_cols_per_thread(d, elem_bytes);  // columns per tile
    long long ncol_total = 0;
    for (int k = 0; k < ninst; ++k) ncol_total += (n[k] + TW - 1) / TW;
    // enough tiles to fill the GPU (152 SMs x 8 CTAs), rows per band a multiple of 64
    const long long target = 152 * 8;
    const long long f = std::max<long long>(1, (target + ncol_total - 1) / std::max<long long>(ncol_total, 1));
    AdjTotals tot{0, 0, 0, 0, 0, 0};
    for (int k = 0; k < ninst; ++k) {
        AdjInst &I = out[k];
        I.m = m[k];
        I.n = n[k];
        I.ncol = (n[k] + TW - 1) / TW;
        const long long maxb = (m[k] + 63) / 64;
        const int nb0 = (int)std::min<long long>(f, maxb);
        int rh = (m[k] + nb0 - 1) / nb0;
        rh = std::min(((rh + 63) / 64) * 64, kAdjBandMax);
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
        I.fin0 = (int)tot.fin_blocks;
        tot.fin_blocks += (m[k] + kFinThreads - 1) / kFinThreads + (n[k] + kFinThreads - 1) / kFinThreads;
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
