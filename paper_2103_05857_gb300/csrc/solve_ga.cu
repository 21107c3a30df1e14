// solve_ga.cu -- one epoch (m block updates) with gap-adaptive block
// sampling (Sec. 4.2, Alg. A.4) on a single instance, one CTA.
//
// Block i is drawn with probability proportional to max(g_i, 0), where g_i is
// the block gap of eq. 11 as last evaluated. The per-row gaps live in global
// memory (FP64, m entries); sums over chunks of 32 rows are kept in shared
// memory. Warp 0 samples: u = draw(seed, 3, k) gives the target u * total;
// a warp scan over contiguous groups of chunk sums finds the chunk, a second
// scan over the chunk's 32 gaps finds the row (first row whose cumulative
// weight exceeds the target). Past 8192 rows the tree has a third level:
// sums of super nodes of 32 chunks, scanned first. After the update of row i its gap is evaluated
// again at the new plan and residual (the line of Alg. A.4 that follows the
// update), and the chunk sum is recomputed from its 32 entries, so no
// rounding accumulates in the sums. Full refreshes of every g_i (every M
// epochs) are certificate passes run by the host between epochs.
//
// Rows cannot be prefetched (the next row depends on this update's gap), so
// each update loads its row of T (and of C when given) directly; the block
// update itself is the one of the dense epoch kernel: one fused reduction
// (argmin, line-search sums, away vertex), the decision of step.cuh, and the
// rank-1 update of the residual held in registers.
//
// The post-update gap is taken in the shifted form
//   g_i = sum_j t_ij (grad_ij - mu) - a_i (min_j grad_ij - mu),
// mu = the pre-update minimum, which equals eq. 11 exactly in real arithmetic
// and avoids the cancellation of its two large terms in FP32.
#include <limits>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "step.cuh"

namespace srot {

namespace {

constexpr int kGaMaxChunks = 256;     // two-level sampling: m <= 8192
constexpr int kGaMaxSupers = 256;     // three-level sampling (32 chunks of 32 rows per super
                                      // node): m <= 262144

// Row drawn by gap-adaptive sampling; run by all 32 lanes of one warp,
// returns the row on every lane.
__device__ inline int ga_sample(const double *g, const double *csum, int m, unsigned long long seed,
                                long long k) {
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nch = (m + 31) >> 5;
    const int L = (nch + 31) >> 5;  // chunks per lane, contiguous
    const uint64_t u64 = sm64_draw(seed, 3, (uint64_t)k);
    double part = 0.0;
    for (int c = lane * L; c < min(nch, lane * L + L); ++c) part += csum[c];
    // inclusive scan over lanes
    double incl = part;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(F, incl, o);
        if (lane >= o) incl += v;
    }
    const double total = __shfl_sync(F, incl, 31);
    if (!(total > 0.0)) return scale_u64(u64, m);
    const double target = (double)(u64 >> 11) * 0x1.0p-53 * total;
    // lane whose group of chunks crosses the target
    unsigned cross = __ballot_sync(F, incl > target && part > 0.0);
    int src, chunk = -1;
    double base;
    if (cross) {
        src = __ffs(cross) - 1;
        base = __shfl_sync(F, incl - part, src);
        if (lane == src) {
            double cum = base;
            for (int c = src * L; c < min(nch, src * L + L); ++c) {
                if (csum[c] > 0.0 && cum + csum[c] > target) { chunk = c; break; }
                cum += csum[c];
            }
            if (chunk < 0) {  // rounding: the last positive chunk of the group
                for (int c = min(nch, src * L + L) - 1; c >= src * L; --c)
                    if (csum[c] > 0.0) { chunk = c; break; }
                cum = base;
                for (int c = src * L; c < chunk; ++c) cum += csum[c];
            } else {
                // cum is the weight before `chunk`
            }
            base = cum;
        }
        chunk = __shfl_sync(F, chunk, src);
        base = __shfl_sync(F, base, src);
    } else {
        // rounding put the target at or past the total: the last positive chunk
        int lastc = -1;
        for (int c = lane * L; c < min(nch, lane * L + L); ++c)
            if (csum[c] > 0.0) lastc = c;
        lastc = __reduce_max_sync(F, lastc + 1) - 1;
        chunk = lastc;
        base = -1.0;  // take the last positive row of the chunk
    }
    if (chunk < 0) return scale_u64(u64, m);  // no positive weight found: uniform
    const int i = chunk * 32 + lane;
    const double w = (i < m && g[i] > 0.0) ? g[i] : 0.0;
    double ci = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(F, ci, o);
        if (lane >= o) ci += v;
    }
    const unsigned hit = base >= 0.0 ? __ballot_sync(F, w > 0.0 && base + ci > target) : 0u;
    if (hit) return chunk * 32 + __ffs(hit) - 1;
    const unsigned pos = __ballot_sync(F, w > 0.0);
    if (!pos) return scale_u64(u64, m);
    return chunk * 32 + (31 - __clz(pos));
}

// Among 32 weights w (one per lane, in order) preceded by weight `base`: the
// first lane whose cumulative weight exceeds `target` (with *before, the
// weight before it), or with base < 0 (or no such lane: rounding put the
// target past the total) the last lane of positive weight (*before = -1).
// -1 if no weight is positive. All 32 lanes; every lane returns the same.
__device__ inline int ga_pick32(double w, double base, double target, double *before) {
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    double ci = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(F, ci, o);
        if (lane >= o) ci += v;
    }
    const unsigned hit = base >= 0.0 ? __ballot_sync(F, w > 0.0 && base + ci > target) : 0u;
    if (hit) {
        const int l = __ffs(hit) - 1;
        *before = base + __shfl_sync(F, ci - w, l);
        return l;
    }
    const unsigned pos = __ballot_sync(F, w > 0.0);
    *before = -1.0;
    return pos ? 31 - __clz(pos) : -1;
}

// Gap-adaptive draw for m > 8192: the same inverse transform over a
// three-level tree of cumulative sums (super nodes of 32 chunks of 32 rows):
// a warp scan over the super sums (contiguous groups per lane) finds the
// super node, a scan over its 32 chunk sums the chunk, a scan over the
// chunk's 32 gaps the row. One warp; returns the row on every lane.
__device__ inline int ga_sample3(const double *g, const double *csum, const double *ssum, int m,
                                 unsigned long long seed, long long k) {
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nch = (m + 31) >> 5;
    const int nsup = (nch + 31) >> 5;
    const int L = (nsup + 31) >> 5;  // super nodes per lane, contiguous
    const uint64_t u64 = sm64_draw(seed, 3, (uint64_t)k);
    double part = 0.0;
    for (int c = lane * L; c < min(nsup, lane * L + L); ++c) part += ssum[c];
    double incl = part;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(F, incl, o);
        if (lane >= o) incl += v;
    }
    const double total = __shfl_sync(F, incl, 31);
    if (!(total > 0.0)) return scale_u64(u64, m);
    const double target = (double)(u64 >> 11) * 0x1.0p-53 * total;
    // the super node: within the lane group that crosses the target
    const unsigned cross = __ballot_sync(F, incl > target && part > 0.0);
    int sup = -1;
    double base = -1.0;
    if (cross) {
        const int src = __ffs(cross) - 1;
        if (lane == src) {
            double cum = incl - part;
            for (int c = src * L; c < min(nsup, src * L + L); ++c) {
                if (ssum[c] > 0.0 && cum + ssum[c] > target) { sup = c; base = cum; break; }
                cum += ssum[c];
            }
            if (sup < 0)  // rounding: the last positive super node of the group
                for (int c = min(nsup, src * L + L) - 1; c >= src * L; --c)
                    if (ssum[c] > 0.0) { sup = c; base = -1.0; break; }
        }
        sup = __shfl_sync(F, sup, src);
        base = __shfl_sync(F, base, src);
    } else {
        int lastc = -1;
        for (int c = lane * L; c < min(nsup, lane * L + L); ++c)
            if (ssum[c] > 0.0) lastc = c;
        sup = __reduce_max_sync(F, lastc + 1) - 1;
    }
    if (sup < 0) return scale_u64(u64, m);
    const int c1 = sup * 32 + lane;
    double before = -1.0;
    const int lc = ga_pick32(c1 < nch ? csum[c1] : 0.0, base, target, &before);
    if (lc < 0) return scale_u64(u64, m);
    const int chunk = sup * 32 + lc;
    const int r = chunk * 32 + lane;
    const double w = (r < m && g[r] > 0.0) ? g[r] : 0.0;
    double unused;
    const int lr = ga_pick32(w, before, target, &unused);
    if (lr < 0) return scale_u64(u64, m);
    return chunk * 32 + lr;
}

template <typename Real, int NT, int G, bool PTS, bool AWAY>
__global__ void __launch_bounds__(NT, 1) k_epoch_ga(EpochArgs<Real> A) {
    using RedT = typename std::conditional<std::is_same<Real, float>::value, RedF, RedD>::type;
    constexpr bool F32 = std::is_same<Real, float>::value;
    constexpr int NW = NT / kWarp;
    constexpr int CPT = 4 * G;
    constexpr int WID = NT * CPT;
    __shared__ __align__(16) Real rowbuf[WID];
    __shared__ RedT red[2][kMaxWarps];
    __shared__ double ssum[kGaMaxSupers];
    __shared__ int sel;
    extern __shared__ double csum[];  // chunk sums: ceil(m / 32)

    const int m = A.in.m, n = A.in.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Real INF = std::numeric_limits<Real>::infinity();
    const Real rho = (Real)A.rho;
    double *g = A.g_store;

    Real q[CPT];
    float qc[F32 ? CPT : 1];
    Real y0[PTS ? CPT : 1], y1[PTS ? CPT : 1], y2[PTS ? CPT : 1];
#pragma unroll
    for (int gg = 0; gg < G; ++gg)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = 4 * gg + e, j = 4 * (tid + NT * gg) + e;
            if constexpr (F32) {
                const double qq = j < n ? A.q[j] : 1e30;
                q[c] = (float)qq;
                qc[c] = j < n ? (float)((double)q[c] - qq) : 0.f;
            } else {
                q[c] = j < n ? A.q[j] : INF;
            }
            if (PTS) {
                y0[c] = j < n ? A.in.Y[(size_t)j * 3 + 0] : Real(0);
                y1[c] = j < n ? A.in.Y[(size_t)j * 3 + 1] : Real(0);
                y2[c] = j < n ? A.in.Y[(size_t)j * 3 + 2] : Real(0);
            }
        }
    // chunk sums of the clamped gaps
    const int nch = (m + 31) >> 5;
    for (int c = warp; c < nch; c += NW) {
        const int i = c * 32 + lane;
        double w = (i < m && g[i] > 0.0) ? g[i] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) csum[c] = w;
    }
    __syncthreads();
    // super-node sums (32 chunks each), for m > 8192
    const bool three = nch > kGaMaxChunks;
    const int nsup = (nch + 31) >> 5;
    if (three) {
        for (int sp = warp; sp < nsup; sp += NW) {
            const int c = sp * 32 + lane;
            double w = c < nch ? csum[c] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            if (lane == 0) ssum[sp] = w;
        }
        __syncthreads();
    }

    const bool sums = (A.variant == SR_OT_BCFW && A.step == SR_OT_ELS) || A.variant == SR_OT_BCAFW;
    const bool cnt = A.variant == SR_OT_BCAFW;
    const int jbase = 4 * tid;
    int par = 0;
    for (int p = 0; p < m; ++p) {
        const long long k = A.k0 + p;
        if (warp == 0) {
            const int i = three ? ga_sample3(g, csum, ssum, m, A.seed, k) : ga_sample(g, csum, m, A.seed, k);
            if (lane == 0) sel = i;
        }
        __syncthreads();
        const int i = sel;
        Real x0 = Real(0), x1 = Real(0), x2 = Real(0);
        if (PTS) {
            x0 = A.in.X[(size_t)i * 3 + 0];
            x1 = A.in.X[(size_t)i * 3 + 1];
            x2 = A.in.X[(size_t)i * 3 + 2];
        }
        const Real ai = A.in.a[i];
        Real *trow = A.T + (size_t)i * n;
        const Real *crow = PTS ? nullptr : A.in.C + (size_t)i * n;
        Real tv[CPT], cs[CPT];
#pragma unroll
        for (int gg = 0; gg < G; ++gg)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 4 * gg + e, j = jbase + 4 * NT * gg + e;
                tv[c] = j < n ? trow[j] : Real(0);
                cs[c] = (!PTS && j < n) ? crow[j] : Real(0);
                rowbuf[j] = tv[c];
            }
        Step<Real> S;
        Real gmin_pre;
        if constexpr (F32) {
            float gmin = INF, gmax = -INF, s1 = 0.f, s2 = 0.f, rsum = 0.f;
            int jmin = jbase, jmax = 0x7FFFFFFF, nnz = 0;
#pragma unroll
            for (int gg = 0; gg < G; ++gg)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = 4 * gg + e, j = jbase + 4 * NT * gg + e;
                    const float t = tv[c];
                    const float cst = PTS ? cost3(x0, x1, x2, y0[c], y1[c], y2[c]) : cs[c];
                    const float gr = cst + q[c];
                    if (gr < gmin) { gmin = gr; jmin = j; }
                    if (sums) {
                        s1 = fmaf(t, gr, s1);
                        s2 = fmaf(t, t, s2);
                    }
                    if (AWAY) {
                        const float ga = t > 0.f ? gr : -INF;
                        if (ga > gmax) { gmax = ga; jmax = j; }
                        if (cnt) { nnz += t > 0.f; rsum += t; }
                    }
                }
            const uint32_t kmax = (jmax == 0x7FFFFFFF) ? 0u : f2key(gmax);
            Red<float> R = block_reduce<AWAY, NW>(red, par, sums, cnt, f2key(gmin), jmin, s1, s2, kmax, jmax, nnz, rsum);
            par ^= 1;
            if (!isfinite(R.gmin)) { if (tid == 0) atomicCAS(A.status, 0, (int)kDevNonFinite); break; }
            const float t_js = rowbuf[R.jmin];
            const float t_v = (AWAY && R.jmax >= 0 && R.jmax < n) ? rowbuf[R.jmax] : 0.f;
            S = decide<float>(R, ai, t_js, t_v, A.variant, A.step, rho, m, k);
            gmin_pre = R.gmin;
            if (tid == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = i;
                A.trace[4 * k + 1] = R.jmin;
                A.trace[4 * k + 2] = trace_vdir((AWAY && R.jmax >= 0 && R.jmax < n) ? R.jmax : -1, S.kind);
                A.trace[4 * k + 3] = __float_as_int(S.gamma);
            }
        } else {
            double gmin = 0.0, gmax = 0.0, s1 = 0.0, s2 = 0.0;
            int jmin = 0x7FFFFFFF, jmax = 0x7FFFFFFF, nnz = 0;
#pragma unroll
            for (int gg = 0; gg < G; ++gg)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = 4 * gg + e, j = jbase + 4 * NT * gg + e;
                    const double t = tv[c];
                    const double cst = PTS ? cost3(x0, x1, x2, y0[c], y1[c], y2[c]) : cs[c];
                    const double gr = dadd(cst, dmul((double)rho, q[c]));
                    if (j < n) {
                        if (jmin == 0x7FFFFFFF || gr < gmin) { gmin = gr; jmin = j; }
                        if (sums) {
                            s1 = fma(t, gr, s1);
                            s2 = fma(t, t, s2);
                        }
                        if (AWAY && t > 0.0) {
                            ++nnz;
                            if (jmax == 0x7FFFFFFF || gr > gmax) { gmax = gr; jmax = j; }
                        }
                    }
                }
            Red<double> R = block_reduce<AWAY, NW>(red, par, sums, cnt, gmin, jmin, s1, s2, gmax, jmax, nnz);
            par ^= 1;
            if (!isfinite(R.gmin)) { if (tid == 0) atomicCAS(A.status, 0, (int)kDevNonFinite); break; }
            const double t_js = rowbuf[R.jmin];
            const double t_v = (AWAY && R.jmax >= 0 && R.jmax < n) ? (double)rowbuf[R.jmax] : 0.0;
            S = decide<double>(R, (double)ai, t_js, t_v, A.variant, A.step, (double)rho, m, k);
            gmin_pre = R.gmin;
            if (tid == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = i;
                A.trace[4 * k + 1] = R.jmin;
                A.trace[4 * k + 2] = trace_vdir((AWAY && R.jmax >= 0 && R.jmax < n) ? R.jmax : -1, S.kind);
                A.trace[4 * k + 3] = __float_as_int((float)S.gamma);
            }
        }
        // ---- update of the row and of the residual -------------------------
        Real tn[CPT];
#pragma unroll
        for (int gg = 0; gg < G; ++gg)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 4 * gg + e, j = jbase + 4 * NT * gg + e;
                const Real t = tv[c];
                tn[c] = S.kind >= 0 ? apply<Real>(S, j, t) : t;
                if (j < n && tn[c] != t) {
                    if constexpr (F32) kahan2(q[c], qc[c], rho * (tn[c] - t));
                    else q[c] = dadd(q[c], dsub(tn[c], t));
                    trow[j] = tn[c];
                }
            }
        // ---- gap of block i at the new plan (Alg. A.4, inner update) -------
        if (A.ga_inner) {
            double gi;
            if constexpr (F32) {
                float gmin = INF, s1 = 0.f;
                int jmin = jbase;
#pragma unroll
                for (int gg = 0; gg < G; ++gg)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 4 * gg + e, j = jbase + 4 * NT * gg + e;
                        const float cst = PTS ? cost3(x0, x1, x2, y0[c], y1[c], y2[c]) : cs[c];
                        const float gr = cst + q[c];
                        if (gr < gmin) { gmin = gr; jmin = j; }
                        s1 = fmaf(tn[c], gr - gmin_pre, s1);
                    }
                Red<float> R = block_reduce<false, NW>(red, par, true, false, f2key(gmin), jmin, s1, 0.f, 0u,
                                                       0x7FFFFFFF, 0);
                par ^= 1;
                gi = (double)R.s1 - (double)ai * ((double)R.gmin - (double)gmin_pre);
            } else {
                double gmin = 0.0, s1 = 0.0;
                int jmin = 0x7FFFFFFF;
#pragma unroll
                for (int gg = 0; gg < G; ++gg)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 4 * gg + e, j = jbase + 4 * NT * gg + e;
                        const double cst = PTS ? cost3(x0, x1, x2, y0[c], y1[c], y2[c]) : cs[c];
                        const double gr = dadd(cst, dmul((double)rho, q[c]));
                        if (j < n) {
                            if (jmin == 0x7FFFFFFF || gr < gmin) { gmin = gr; jmin = j; }
                            s1 = fma(tn[c], gr - gmin_pre, s1);
                        }
                    }
                Red<double> R = block_reduce<false, NW>(red, par, true, false, gmin, jmin, s1, 0.0, 0.0,
                                                        0x7FFFFFFF, 0);
                par ^= 1;
                gi = R.s1 - (double)ai * (R.gmin - gmin_pre);
            }
            if (warp == 0) {
                const int c0 = i >> 5;
                const int r = c0 * 32 + lane;
                double w = r == i ? gi : ((r < m) ? g[r] : 0.0);
                if (lane == (i & 31)) g[i] = gi;
                w = w > 0.0 ? w : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                if (lane == 0) csum[c0] = w;
                if (three) {  // its super node's sum, from its 32 chunk sums
                    __syncwarp();
                    const int c = (c0 >> 5) * 32 + lane;
                    double w2 = c < nch ? csum[c] : 0.0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) w2 += __shfl_xor_sync(0xffffffffu, w2, o);
                    if (lane == 0) ssum[c0 >> 5] = w2;
                }
            }
        }
        __syncthreads();  // sampling reads csum and g; rowbuf is rewritten
    }
    // running residual back to global memory for the next epoch
    __syncthreads();
#pragma unroll
    for (int gg = 0; gg < G; ++gg)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = 4 * gg + e, j = 4 * (tid + NT * gg) + e;
            if (j < n) {
                if constexpr (F32) A.q[j] = (double)q[c] - (double)qc[c];
                else A.q[j] = q[c];
            }
        }
}

template <typename Real, int NT, int G, bool PTS, bool AWAY>
void launch_ga_kernel(const EpochArgs<Real> &A, cudaStream_t st) {
    auto kern = k_epoch_ga<Real, NT, G, PTS, AWAY>;
    const size_t dyn = sizeof(double) * (size_t)((A.in.m + 31) / 32);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (32 * kGaMaxSupers)));
        attr_set = true;
    }
    kern<<<1, NT, dyn, st>>>(A);
}

template <typename Real, int NT, int G>
void launch_ga_shape(const EpochArgs<Real> &A, cudaStream_t st) {
    const bool pts = A.in.cost_mode == kCostPts3;
    const bool away = A.variant == SR_OT_BCAFW || A.variant == SR_OT_BCPFW;
    if (pts) {
        if (away) launch_ga_kernel<Real, NT, G, true, true>(A, st);
        else launch_ga_kernel<Real, NT, G, true, false>(A, st);
    } else {
        if (away) launch_ga_kernel<Real, NT, G, false, true>(A, st);
        else launch_ga_kernel<Real, NT, G, false, false>(A, st);
    }
}

}  // namespace

int epoch_ga_max_m() { return 32 * 32 * kGaMaxSupers; }

template <>
bool launch_epoch_ga<float>(const EpochArgs<float> &A, cudaStream_t st) {
    const int n = A.in.n;
    if (A.in.m > epoch_ga_max_m()) return false;
    if (n <= 512 * 4) launch_ga_shape<float, 512, 1>(A, st);
    else if (n <= 512 * 8) launch_ga_shape<float, 512, 2>(A, st);
    else if (n <= 512 * 16) launch_ga_shape<float, 512, 4>(A, st);
    else return false;
    return true;
}

template <>
bool launch_epoch_ga<double>(const EpochArgs<double> &A, cudaStream_t st) {
    const int n = A.in.n;
    if (A.in.m > epoch_ga_max_m()) return false;
    if (n <= 256 * 4) launch_ga_shape<double, 256, 1>(A, st);
    else if (n <= 256 * 8) launch_ga_shape<double, 256, 2>(A, st);
    else return false;
    return true;
}

}  // namespace srot
