// reduce.cuh -- the fused block reduction of one block update (argmin,
// line-search dot products, away-vertex argmax, active count) shared by the
// dense epoch kernels.
#pragma once

#include "common.cuh"
#include "step.cuh"

namespace srot {

constexpr int kMaxWarps = 16;

struct RedF {
    uint32_t kmin; int jmin; float s1; float s2;
    uint32_t kmax; int jmax; int nnz; float rs;  // rs: row sum (away steps)
};
struct RedD {
    double gmin; double s1; double s2; double gmax;
    int jmin; int jmax; int nnz; int pad;
};

// ---------------------------------------------------------------------------
// Fused block reduction. `par` selects one of two smem slot arrays so that a
// fast warp writing the next update's partials never overwrites slots a slow
// warp is still reading. `sums` (line-search dot products) and `cnt`
// (active-atom count) are block-uniform flags: reductions a step rule does
// not need are skipped.
// ---------------------------------------------------------------------------
template <bool AWAY, int NW>
__device__ inline Red<float> block_reduce(RedF (*red)[kMaxWarps], int par, bool sums, bool cnt,
                                          uint32_t kmin, int jmin, float s1, float s2,
                                          uint32_t kmax, int jmax, int nnz, float rs = 0.f) {
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t wk = __reduce_min_sync(F, kmin);
    int wj = __reduce_min_sync(F, kmin == wk ? jmin : 0x7FFFFFFF);
    if (sums) {
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
    }
    uint32_t wkx = 0; int wjx = 0x7FFFFFFF, wn = 0;
    if (AWAY) {
        wkx = __reduce_max_sync(F, kmax);
        wjx = __reduce_min_sync(F, kmax == wkx ? jmax : 0x7FFFFFFF);
        if (cnt) {
            wn = __reduce_add_sync(F, nnz);
            rs = warp_sum(rs);
        }
    }
    if (lane == 0) red[par][warp] = RedF{wk, wj, s1, s2, wkx, wjx, wn, rs};
    __syncthreads();
    RedF e = lane < NW ? red[par][lane] : RedF{0xFFFFFFFFu, 0x7FFFFFFF, 0.f, 0.f, 0u, 0x7FFFFFFF, 0, 0.f};
    wk = __reduce_min_sync(F, e.kmin);
    wj = __reduce_min_sync(F, e.kmin == wk ? e.jmin : 0x7FFFFFFF);
    Red<float> r;
    r.gmin = key2f(wk);
    r.jmin = wj;
    r.s1 = sums ? warp_sum(e.s1) : 0.f;
    r.s2 = sums ? warp_sum(e.s2) : 0.f;
    if (AWAY) {
        wkx = __reduce_max_sync(F, e.kmax);
        r.jmax = __reduce_min_sync(F, e.kmax == wkx ? e.jmax : 0x7FFFFFFF);
        r.gmax = key2f(wkx);
        r.nnz = cnt ? __reduce_add_sync(F, e.nnz) : 0;
        r.rs = cnt ? warp_sum(e.rs) : 0.f;
    } else {
        r.gmax = 0.f; r.jmax = -1; r.nnz = 0; r.rs = 0.f;
    }
    return r;
}

__device__ inline void dmin_pair(double &g, int &j, double og, int oj) {
    if (oj != 0x7FFFFFFF && (j == 0x7FFFFFFF || og < g || (og == g && oj < j))) { g = og; j = oj; }
}
__device__ inline void dmax_pair(double &g, int &j, double og, int oj) {
    if (oj != 0x7FFFFFFF && (j == 0x7FFFFFFF || og > g || (og == g && oj < j))) { g = og; j = oj; }
}

template <bool AWAY, int NW>
__device__ inline Red<double> block_reduce(RedD (*red)[kMaxWarps], int par, bool sums, bool cnt,
                                           double gmin, int jmin, double s1, double s2,
                                           double gmax, int jmax, int nnz) {
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dmin_pair(gmin, jmin, __shfl_xor_sync(F, gmin, o), __shfl_xor_sync(F, jmin, o));
        if (sums) {
            s1 += __shfl_xor_sync(F, s1, o);
            s2 += __shfl_xor_sync(F, s2, o);
        }
        if (AWAY) {
            dmax_pair(gmax, jmax, __shfl_xor_sync(F, gmax, o), __shfl_xor_sync(F, jmax, o));
            if (cnt) nnz += __shfl_xor_sync(F, nnz, o);
        }
    }
    if (lane == 0) red[par][warp] = RedD{gmin, s1, s2, gmax, jmin, jmax, nnz, 0};
    __syncthreads();
    RedD e = lane < NW ? red[par][lane] : RedD{0.0, 0.0, 0.0, 0.0, 0x7FFFFFFF, 0x7FFFFFFF, 0, 0};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dmin_pair(e.gmin, e.jmin, __shfl_xor_sync(F, e.gmin, o), __shfl_xor_sync(F, e.jmin, o));
        if (sums) {
            e.s1 += __shfl_xor_sync(F, e.s1, o);
            e.s2 += __shfl_xor_sync(F, e.s2, o);
        }
        if (AWAY) {
            dmax_pair(e.gmax, e.jmax, __shfl_xor_sync(F, e.gmax, o), __shfl_xor_sync(F, e.jmax, o));
            if (cnt) e.nnz += __shfl_xor_sync(F, e.nnz, o);
        }
    }
    Red<double> r;
    r.gmin = e.gmin; r.jmin = e.jmin; r.s1 = e.s1; r.s2 = e.s2;
    r.gmax = e.gmax; r.jmax = AWAY ? e.jmax : -1; r.nnz = e.nnz;
    r.rs = -1.0;  // the FP64 path keeps the oracle's form of the away step
    return r;
}

// value hi - lo += d (Kahan), with round-to-nearest intrinsics so it is never
// contracted or reordered
__device__ inline void kahan2(float &hi, float &lo, float d) {
    float y = __fsub_rn(d, lo);
    float t = __fadd_rn(hi, y);
    lo = __fsub_rn(__fsub_rn(t, hi), y);
    hi = t;
}

}  // namespace srot
