// solve_f64w.cu -- one epoch of FP64 BCFW (Alg. 1; decay rule or exact line
// search, eq. 8) on a single instance of width n <= 512, run by ONE warp.
//
// GB300's FP64 pipe is a small fraction of its FP32 rate, and each FP64
// instruction on the update chain costs far more than its FP32 counterpart.
// So this kernel keeps FP64 arithmetic to the few entries whose exact value
// decides something, and stays bit-identical to a plain FP64 reference:
//   - the argmin of grad_ij = C_ij + rho r_j (eq. 7, ties to the smallest j)
//     is screened in FP32: with c = fl32(C_ij), p = fl32(rho r_j) and
//     g = fl32(c + p), the exact FP64 gradient lies within
//     e = 4 u (|c| + |p|) + 2^-120 of g (u = 2^-24: one rounding each of C,
//     rho r and the sum, a factor 2 to spare; the absolute term covers
//     subnormal magnitudes). With U the smallest g + e of the row, a
//     column with g - e > U cannot be the exact minimum, so only the columns
//     with g - e <= U -- one or two -- get their gradient in FP64
//     (__dadd_rn, the reference's operation), and the exact (value, index)
//     minimum is taken over them (a bound that is not a number, for values
//     beyond the FP32 range, keeps its column a candidate);
//   - the plan row is updated only where it is non-zero (and at j*), tested
//     on the bit pattern, and rho r_j is recomputed in FP64 only where r_j
//     changed;
//   - an FP64 instruction occupies the pipe for about 60 clocks for the whole
//     warp, however few lanes take part, so each lane keeps a bit mask of its
//     candidates and of its non-zero plan entries, and the lanes work through
//     their masks together: every FP64 operation is issued once per round,
//     and the rounds are as many as the most entries one lane holds (one,
//     as a rule), not one per column slot;
//   - with the decay rule, when the screen leaves a single candidate it is
//     the exact minimum and no FP64 operation is needed for the LMO at all;
//   - the step of the next 32 updates (gamma, 1 - gamma, gamma a_i) is
//     computed one per lane ahead of use;
//   - the decay step 2m/(k+2m) comes from a table the lanes fill 32 updates
//     at a time, so no FP64 division sits on the chain;
//   - one warp, no block barrier: every reduction is a warp reduction.
// Every FP64 value is the same IEEE-754 operation, in the same order, as the
// plain definition of the step (__dadd_rn / __dmul_rn / __dsub_rn /
// __ddiv_rn), so the decay-rule trajectory equals that of an FP64 reference
// written the same way, bit for bit.
//
// Lane l owns the quads j = 4 (l + 32 g) + e, g < G, e < 4 (128-bit shared
// loads). Rows of T, of C and of its FP32 rounding are streamed into a ring
// kF64wRing - 2 updates ahead by the lanes that own their columns; the
// residual state (r_j, rho r_j, fl32(rho r_j)) lives in shared memory. A row
// that repeats within the window (uniform order) is read again from global
// memory, where it was stored.
#include <climits>
#include <limits>

#include "common.cuh"
#include "internal.h"
#include "step.cuh"

namespace srot {

namespace {

constexpr int kF64wRing = 6;  // ring slots: rows streamed kF64wRing - 2 updates ahead

__device__ inline void cpa16(void *dst, const void *src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src));
}
__device__ inline void cpa8(void *dst, const void *src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src));
}
__device__ inline void cpa4(void *dst, const void *src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src));
}
__device__ inline void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Order-preserving unsigned image of a double (+0 and -0 map to the same
// key, as they compare equal).
__device__ inline unsigned long long d2key(double x) {
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if (u == 0x8000000000000000ull) u = 0ull;
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ inline double key2d(unsigned long long k) {
    const unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)u);
}
__device__ inline bool nonzero_bits(double x) { return (__double_as_longlong(x) << 1) != 0; }
__device__ inline double warp_dsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = dadd(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// FP32 rounding of the cost, streamed for the argmin screen.
__global__ void k_round_cost(const double *__restrict__ C, float *__restrict__ C32, size_t count) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        C32[e] = __double2float_rn(C[e]);
}

}  // namespace

template <int G>
__global__ void __launch_bounds__(32, 1) k_epoch_f64w(EpochArgs<double> A) {
    constexpr int CPL = 4 * G;         // columns per lane: G quads
    constexpr int WID = 128 * G;       // padded row width
    constexpr int D = kF64wRing - 2;   // rows streamed D updates ahead
    constexpr int SLOT = 2 * WID + WID / 2;  // doubles per slot: T row, C row, FP32 C row
    constexpr unsigned FULL = 0xffffffffu;
    constexpr float kScreen = 4.0f * 0x1.0p-24f;
    extern __shared__ __align__(16) unsigned char smem[];
    double *ring = reinterpret_cast<double *>(smem);      // kF64wRing x [T | C | C32]
    double *rcol = ring + (size_t)kF64wRing * SLOT;       // r_j
    double *rrs = rcol + WID;                             // rho r_j
    float *rfs = reinterpret_cast<float *>(rrs + WID);    // fl32(rho r_j)
    const int m = A.in.m, n = A.in.n;
    const int lane = threadIdx.x;
    const double rho = A.rho;
    const bool dec = A.step == SR_OT_DEC;
    // 16-byte copies: T and C rows (doubles) when n is even and the rows
    // aligned (A.vec); the FP32 cost quads only when n is also a multiple of
    // 4, else as two 8-byte halves
    const bool vec = A.vec;
    const bool vec32 = vec && (n % 4) == 0;
    const float FINF = std::numeric_limits<float>::infinity();
    auto tslot = [&](int s) { return ring + (size_t)s * SLOT; };
    auto cslot = [&](int s) { return ring + (size_t)s * SLOT + WID; };
    auto fslot = [&](int s) { return reinterpret_cast<float *>(ring + (size_t)s * SLOT + 2 * WID); };
    auto col = [&](int c) { return 4 * (lane + 32 * (c >> 2)) + (c & 3); };

    // residual state per column; padding columns get +inf (never a
    // candidate) and zero plan and cost entries in every slot
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int j = col(c);
        const double r = j < n ? A.q[j] : 0.0;
        rcol[j] = r;
        rrs[j] = j < n ? dmul(rho, r) : std::numeric_limits<double>::infinity();
        rfs[j] = j < n ? __double2float_rn(rrs[j]) : FINF;
        if (j >= n)
            for (int s = 0; s < kF64wRing; ++s) {
                tslot(s)[j] = 0.0;
                cslot(s)[j] = 0.0;
                fslot(s)[j] = 0.f;
            }
    }

    auto row_of = [&](int p) -> int {
        if (p >= m) return -1;
        if (A.order == SR_OT_CYCLIC) return p;
        if (A.order == SR_OT_PERMUTE) return A.perm[p];
        return scale_u64(sm64_draw(A.seed, 2, (uint64_t)(A.k0 + p)), m);
    };
    auto fetch_async = [&](int i, int s) {
        const double *tsrc = A.T + (size_t)i * n;
        const double *csrc = A.in.C + (size_t)i * n;
        const float *fsrc = A.C32 + (size_t)i * n;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j0 = 4 * (lane + 32 * g);
            if (vec && j0 + 3 < n) {
                cpa16(tslot(s) + j0, tsrc + j0);
                cpa16(tslot(s) + j0 + 2, tsrc + j0 + 2);
                cpa16(cslot(s) + j0, csrc + j0);
                cpa16(cslot(s) + j0 + 2, csrc + j0 + 2);
                if (vec32) {
                    cpa16(fslot(s) + j0, fsrc + j0);
                } else {
                    cpa8(fslot(s) + j0, fsrc + j0);
                    cpa8(fslot(s) + j0 + 2, fsrc + j0 + 2);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j0 + e < n) {
                        cpa8(tslot(s) + j0 + e, tsrc + j0 + e);
                        cpa8(cslot(s) + j0 + e, csrc + j0 + e);
                        cpa4(fslot(s) + j0 + e, fsrc + j0 + e);
                    }
            }
        }
    };
    auto fetch_sync = [&](int i, int s) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int j = col(c);
            if (j < n) {
                tslot(s)[j] = A.T[(size_t)i * n + j];
                cslot(s)[j] = A.in.C[(size_t)i * n + j];
                fslot(s)[j] = A.C32[(size_t)i * n + j];
            }
        }
    };

    // rq[t]: row of update p + t; aq[t]: that row travels by cp.async
    int rq[D + 2];
    bool aq[D + 1];
#pragma unroll
    for (int t = 0; t < D + 2; ++t) rq[t] = row_of(t);
#pragma unroll
    for (int t = 0; t < D; ++t) {
        bool ok = rq[t] >= 0;
#pragma unroll
        for (int u = 0; u < t; ++u) ok = ok && rq[t] != rq[u];
        aq[t] = ok;
        if (ok) fetch_async(rq[t], t % kF64wRing);
        cpa_commit();
    }
    __syncwarp();
    // the step of the next 32 updates, one per lane: gamma (decay rule),
    // 1 - gamma and gamma a_i of that update's row, and a_i
    double tg = 0.0, tcoef = 0.0, tadd = 0.0, ta = 0.0;
    int i_prev = -1;
    for (int p = 0; p < m; ++p) {
        const long long k = A.k0 + p;
        const int i = rq[0];
        const int s = p % kF64wRing;
        {
            bool ok = rq[D] >= 0 && rq[D] != i_prev;
#pragma unroll
            for (int u = 0; u < D; ++u) ok = ok && rq[D] != rq[u];
            aq[D] = ok;
            if (ok) fetch_async(rq[D], (p + D) % kF64wRing);
            cpa_commit();
        }
        const int r_far = row_of(p + D + 2);
        if ((p & 31) == 0) {
            const int rl = row_of(p + lane);
            ta = rl >= 0 ? A.in.a[rl] : 0.0;
            if (dec) {
                const double twom = 2.0 * (double)m;
                tg = __ddiv_rn(twom, dadd((double)(k + lane), twom));
                tcoef = dsub(1.0, tg);
                tadd = dmul(tg, ta);
            }
        }
        const int tl = p & 31;
        const double ac = __shfl_sync(FULL, ta, tl);
        if (aq[0]) cpa_wait<D>();
        else fetch_sync(i, s);
        __syncwarp();
        const double *trs = tslot(s);
        const double *crs = cslot(s);
        const float *frs = fslot(s);

        // ---- argmin (eq. 7): FP32 screen ----------------------------------
        float lo[CPL];
        float hmin = FINF;
        unsigned supm = 0;  // this lane's non-zero plan entries (bit c)
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j0 = 4 * (lane + 32 * g);
            const float4 cf4 = *reinterpret_cast<const float4 *>(frs + j0);
            const float4 pf4 = *reinterpret_cast<const float4 *>(rfs + j0);
            const longlong2 t01 = *reinterpret_cast<const longlong2 *>(trs + j0);
            const longlong2 t23 = *reinterpret_cast<const longlong2 *>(trs + j0 + 2);
            const float cf[4] = {cf4.x, cf4.y, cf4.z, cf4.w};
            const float pf[4] = {pf4.x, pf4.y, pf4.z, pf4.w};
            const long long tb[4] = {t01.x, t01.y, t23.x, t23.y};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float gs = __fadd_rn(cf[e], pf[e]);
                const float er = kScreen * (fabsf(cf[e]) + fabsf(pf[e])) + 0x1.0p-120f;
                lo[4 * g + e] = gs - er;
                hmin = fminf(hmin, gs + er);
                if ((tb[e] << 1) != 0) supm |= 1u << (4 * g + e);
            }
        }
        const float U = key2f(__reduce_min_sync(FULL, f2key(hmin)));
        // candidates (a bound that is not a number, for values beyond the
        // FP32 range, keeps its column a candidate)
        unsigned cand = 0;
#pragma unroll
        for (int c = 0; c < CPL; ++c)
            if (col(c) < n && !(lo[c] > U)) cand |= 1u << c;
        const int ncand = __reduce_add_sync(FULL, __popc(cand));
        int js;
        double gmin = 0.0;
        if (ncand == 1 && dec) {
            // one candidate: it is the exact minimum, and the decay rule needs
            // no gradient value
            js = __reduce_max_sync(FULL, cand ? col(__ffs(cand) - 1) : -1);
        } else {
            // ---- exact FP64 gradient on the candidates ---------------------
            unsigned long long kmin = ~0ull;
            int jmin = INT_MAX;
            unsigned mine = cand;
            while (__any_sync(FULL, mine != 0)) {
                if (mine) {
                    const int c = __ffs(mine) - 1;
                    mine &= mine - 1;
                    const int j = col(c);
                    const unsigned long long kk = d2key(dadd(crs[j], rrs[j]));
                    if (kk < kmin || (kk == kmin && j < jmin)) { kmin = kk; jmin = j; }
                }
            }
            const unsigned hi = (unsigned)(kmin >> 32), lw = (unsigned)kmin;
            const unsigned whi = __reduce_min_sync(FULL, hi);
            const unsigned wlo = __reduce_min_sync(FULL, hi == whi ? lw : 0xFFFFFFFFu);
            js = __reduce_min_sync(FULL, (hi == whi && lw == wlo) ? jmin : INT_MAX);
            const unsigned long long wk = ((unsigned long long)whi << 32) | wlo;
            if (js == INT_MAX || wk >= 0xFFF0000000000000ull) js = INT_MAX;  // not finite
            else gmin = key2d(wk);
        }
        if (js == INT_MAX || (ncand == 1 && dec && !(U < FINF))) {  // no finite minimum
            if (lane == 0) atomicCAS(A.status, 0, (int)kDevNonFinite);
            break;
        }
        const double t_js = trs[js];
        // ---- step (Alg. 1): decay rule or exact line search ----------------
        double gam, coef, add;
        const bool move = (__double_as_longlong(ac) << 1) != 0;  // a_i > 0 (weights are >= 0)
        if (dec) {
            gam = __shfl_sync(FULL, tg, tl);
            coef = __shfl_sync(FULL, tcoef, tl);
            add = __shfl_sync(FULL, tadd, tl);
        } else {
            // sum_j t_ij grad_ij and sum_j t_ij^2 over the support
            double s1 = 0.0, s2 = 0.0;
            unsigned mine = supm;
            while (__any_sync(FULL, mine != 0)) {
                if (mine) {
                    const int c = __ffs(mine) - 1;
                    mine &= mine - 1;
                    const int j = col(c);
                    const double t = trs[j];
                    s1 = fma(t, dadd(crs[j], rrs[j]), s1);
                    s2 = fma(t, t, s2);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s1 = dadd(s1, __shfl_xor_sync(FULL, s1, o));
                s2 = dadd(s2, __shfl_xor_sync(FULL, s2, o));
            }
            const double g_fw = s1 - ac * gmin;
            double dd = (s2 - t_js * t_js) + (ac - t_js) * (ac - t_js);
            gam = line_search<double>(g_fw, dd > 0.0 ? dd : 0.0, rho, 1.0);
            coef = dsub(1.0, gam);
            add = dmul(gam, ac);
        }
        if (move) {
            // the row's support and j*: each lane its own columns, each
            // FP64 operation issued once per round
            double *trow = A.T + (size_t)i * n;
            unsigned mine = supm;
            if (lane == ((js >> 2) & 31)) mine |= 1u << (4 * (js >> 7) + (js & 3));  // j* = col(that bit)
            while (__any_sync(FULL, mine != 0)) {
                if (mine) {
                    const int c = __ffs(mine) - 1;
                    mine &= mine - 1;
                    const int j = col(c);
                    const double t = trs[j];
                    double tn = dmul(coef, t);
                    if (j == js) tn = dadd(tn, add);
                    if (__double_as_longlong(tn) != __double_as_longlong(t)) {
                        const double r = dadd(rcol[j], dsub(tn, t));
                        const double rr = dmul(rho, r);
                        rcol[j] = r;
                        rrs[j] = rr;
                        rfs[j] = __double2float_rn(rr);
                        trow[j] = tn;
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0 && A.trace && k < A.trace_cap) {
            A.trace[4 * k] = i;
            A.trace[4 * k + 1] = js;
            A.trace[4 * k + 2] = trace_vdir(-1, 0);  // BCFW: toward the LMO vertex
            A.trace[4 * k + 3] = __float_as_int(move ? (float)gam : 0.f);
        }
        // ---- advance the pipeline -------------------------------------------
        i_prev = i;
#pragma unroll
        for (int t = 0; t < D + 1; ++t) rq[t] = rq[t + 1];
        rq[D + 1] = r_far;
#pragma unroll
        for (int t = 0; t < D; ++t) aq[t] = aq[t + 1];
    }
    cpa_wait<0>();
    __syncwarp();
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int j = col(c);
        if (j < n) A.q[j] = rcol[j];
    }
}

template <int G>
static void launch_f64w(const EpochArgs<double> &A, cudaStream_t st) {
    constexpr size_t smem = ((size_t)kF64wRing * (2 * 128 * G + 64 * G) + 2 * 128 * G) * sizeof(double) +
                            (size_t)128 * G * sizeof(float);
    auto kern = k_epoch_f64w<G>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    kern<<<1, 32, smem, st>>>(A);
}

int epoch_f64w_max_n() { return 512; }

void launch_round_cost(const double *C, float *C32, size_t count, cudaStream_t st) {
    const int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 8);
    k_round_cost<<<blocks, 256, 0, st>>>(C, C32, count);
}

bool launch_epoch_f64w(const EpochArgs<double> &A, cudaStream_t st) {
    if (A.variant != SR_OT_BCFW || A.in.cost_mode != kCostGiven || A.order == SR_OT_GAP_ADAPTIVE) return false;
    if (A.resume_in || !A.C32) return false;
    const int n = A.in.n;
    if (n <= 128) launch_f64w<1>(A, st);
    else if (n <= 256) launch_f64w<2>(A, st);
    else if (n <= 512) launch_f64w<4>(A, st);
    else return false;
    return true;
}

}  // namespace srot
