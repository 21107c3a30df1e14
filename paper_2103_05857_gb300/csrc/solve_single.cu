// solve_single.cu -- one epoch (m block updates) of BCFW / BCAFW / BCPFW on a
// single instance, run by one 512-thread CTA that keeps the running residual
// on chip.
//
// Per block update (Alg. 1; Alg. A.2; Alg. A.3), for row i:
//   grad_ij = C_ij + rho r_j                              (Sec. 3.1)
//   j*      = argmin_j grad_ij, ties to the smallest j     (eq. 7)
//   v       = argmax over active atoms {j : t_ij > 0}      (away vertex, Sec. 4.1)
//   step    = decay 2m/(k+2m) or exact line search          (eq. 8, eq. 10)
//   t_i    <- t_i + gamma d;  r_j += delta t_ij             (rank-1 update of s)
//
// Layout. Thread `tid` owns columns j = tid + 512 c, c < CPT: it keeps the
// residual of those columns (FP32: q = rho r; FP64: r) and, for the d = 3
// point cost, the target points y_j in registers for the whole epoch. Rows
// of T (and of C when it is given) are streamed into a 3-slot shared-memory
// ring by cp.async, two rows ahead of the update that needs them. Every
// thread copies only its own columns; slots are never written in place, and
// the slot refilled during update p (for update p+2) was last read during
// update p-2, which every thread finished before the barrier of update p-1.
// So the one barrier per update (inside the block reduction) is the only
// synchronisation. A row that repeats one of the three rows before it
// (uniform order) is loaded synchronously from global memory, where its
// owner thread stored it, when its update starts. x_i, a_i and the row
// indices travel through a register pipeline two updates ahead.
//
// Reduction. One fused block reduction per update carries the argmin (value,
// index), sum_j t_ij grad_ij and sum_j t_ij^2 (line search), and for away /
// pairwise steps the argmax over active atoms and the active-atom count.
// FP32 keys are order-preserving uint32 images of the gradient, reduced with
// redux.sync; FP64 uses (value, index) shuffles.
//
// FP64 arithmetic uses __dadd_rn/__dmul_rn/__dsub_rn/__ddiv_rn in the order of
// the plain definition, so the decay-rule trajectory (argmin sequence and
// plan) is reproducible bit for bit by an FP64 reference written the same way.
#include <limits>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "step.cuh"

namespace srot {

constexpr int kSmemMax = 227 * 1024;

__device__ inline void cp_async(void *smem_dst, const void *gsrc, int bytes) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc));
}
__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_wait_groups() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
__device__ inline void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ inline void cp_async16(void *smem_dst, const void *gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}

// ---------------------------------------------------------------------------
// The epoch kernel. NT threads; thread tid owns the CPT = 4G columns
// j = 4 (tid + NT g) + e, g < G, e < 4 (quads, so that rows move by 16-byte
// copies and 128-bit shared loads). Rows are padded to NT*CPT columns: padding
// columns carry t = 0 and residual +inf, so they are never the argmin nor
// active, and the compute loops need no bounds checks.
// ---------------------------------------------------------------------------
template <typename Real, int NT, int G, bool PTS, bool AWAY, int RING>
__global__ void __launch_bounds__(NT, 1) k_epoch(EpochArgs<Real> A) {
    using RedT = typename std::conditional<std::is_same<Real, float>::value, RedF, RedD>::type;
    constexpr int NW = NT / kWarp;
    constexpr int CPT = 4 * G;
    constexpr int WID = NT * CPT;                 // padded row width
    constexpr int SLOT = WID * (PTS ? 1 : 2);     // [T row][C row if given]
    constexpr int D = RING - 2;                   // rows streamed D updates ahead
    extern __shared__ __align__(16) unsigned char smem[];
    Real *ring = reinterpret_cast<Real *>(smem);
    RedT(*red)[kMaxWarps] = reinterpret_cast<RedT(*)[kMaxWarps]>(ring + (size_t)RING * SLOT);
    const int m = A.in.m, n = A.in.n;
    const int tid = threadIdx.x;
    const bool vec = A.vec;
    const Real INF = std::numeric_limits<Real>::infinity();

    // Running residual in registers: FP64 path r; FP32 path rho*r as a
    // compensated pair (q, qc), value q - qc, so that many small updates of a
    // large entry (column 0 holds all the mass at the start) do not accumulate
    // FP32 rounding; the gradient uses q. Padding columns get a huge finite
    // residual: never the argmin, and t * grad stays 0 there.
    constexpr bool F32 = std::is_same<Real, float>::value;
    Real q[CPT];
    float qc[F32 ? CPT : 1];
    Real y0[PTS ? CPT : 1], y1[PTS ? CPT : 1], y2[PTS ? CPT : 1];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = 4 * g + e, j = 4 * (tid + NT * g) + e;
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
            if (j >= n)
                for (int s = 0; s < RING; ++s) {
                    ring[(size_t)s * SLOT + j] = Real(0);
                    if (!PTS) ring[(size_t)s * SLOT + WID + j] = Real(0);
                }
        }
    const Real rho = (Real)A.rho;
    const int order = A.order;
    const bool sums = (A.variant == SR_OT_BCFW && A.step == SR_OT_ELS) || A.variant == SR_OT_BCAFW;
    const bool cnt = A.variant == SR_OT_BCAFW;

    auto row_of = [&](int p) -> int {
        if (p >= m) return -1;
        if (order == SR_OT_CYCLIC) return p;
        if (order == SR_OT_PERMUTE) return A.perm[p];
        return scale_u64(sm64_draw(A.seed, 2, (uint64_t)(A.k0 + p)), m);
    };
    // Copy (async) this thread's columns of row i into slot s.
    auto fetch_async = [&](int i, int s) {
        Real *dst = ring + (size_t)s * SLOT;
        const Real *src = A.T + (size_t)i * n;
        const Real *csrc = PTS ? nullptr : A.in.C + (size_t)i * n;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j0 = 4 * (tid + NT * g);
            if (vec && j0 + 3 < n) {
#pragma unroll
                for (int h = 0; h < (int)sizeof(Real) / 4; ++h) {
                    cp_async16(dst + j0 + h * (16 / sizeof(Real)), src + j0 + h * (16 / sizeof(Real)));
                    if (!PTS) cp_async16(dst + WID + j0 + h * (16 / sizeof(Real)), csrc + j0 + h * (16 / sizeof(Real)));
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j0 + e < n) {
                        cp_async(dst + j0 + e, src + j0 + e, sizeof(Real));
                        if (!PTS) cp_async(dst + WID + j0 + e, csrc + j0 + e, sizeof(Real));
                    }
            }
        }
    };
    // Synchronous load of this thread's columns of row i into slot s.
    auto fetch_sync = [&](int i, int s) {
        Real *dst = ring + (size_t)s * SLOT;
        const Real *src = A.T + (size_t)i * n;
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * (tid + NT * g) + e;
                if (j < n) {
                    dst[j] = src[j];
                    if (!PTS) dst[WID + j] = A.in.C[(size_t)i * n + j];
                }
            }
    };
    auto load_xa = [&](int i, Real &x0, Real &x1, Real &x2, Real &ai) {
        if (i < 0) return;
        if (PTS) {
            x0 = A.in.X[(size_t)i * 3 + 0];
            x1 = A.in.X[(size_t)i * 3 + 1];
            x2 = A.in.X[(size_t)i * 3 + 2];
        }
        ai = A.in.a[i];
    };

    const bool prefetchable = (order == SR_OT_CYCLIC || order == SR_OT_PERMUTE || order == SR_OT_UNIFORM);
    // Pipeline: rq[t] = row of update p+t (t <= D+1); aq[t] = that row travels
    // by cp.async (t < D). A row that repeats one of the rows of updates
    // p-1 .. p+D-1 is loaded synchronously when its update starts.
    // A continuation launch starts where the sparse kernel stopped (or does
    // nothing when it finished the epoch).
    int p0 = 0;
    if (A.resume_in) {
        p0 = *A.resume_in;
        if (p0 < 0) return;
    }
    int rq[D + 2];
    bool aq[D + 1];
#pragma unroll
    for (int t = 0; t < D + 2; ++t) rq[t] = row_of(p0 + t);
#pragma unroll
    for (int t = 0; t < D; ++t) {
        bool ok = prefetchable && rq[t] >= 0;
#pragma unroll
        for (int u = 0; u < t; ++u) ok = ok && rq[t] != rq[u];
        aq[t] = ok;
        if (ok) fetch_async(rq[t], (p0 + t) % RING);
        cp_commit();
    }
    Real x0c = Real(0), x1c = Real(0), x2c = Real(0), ac = Real(0);
    load_xa(rq[0], x0c, x1c, x2c, ac);
    int i_prev = -1;
    int par = 0;
    const int jbase = 4 * tid;
    for (int p = p0; p < m; ++p) {
        const long long k = A.k0 + p;
        const int i = rq[0];
        Real *slot = ring + (size_t)(p % RING) * SLOT;
        {
            bool ok = prefetchable && rq[D] >= 0 && rq[D] != i_prev;
#pragma unroll
            for (int u = 0; u < D; ++u) ok = ok && rq[D] != rq[u];
            aq[D] = ok;
            if (ok) fetch_async(rq[D], (p + D) % RING);
            cp_commit();
        }
        const int r_far = row_of(p + D + 2);
        Real x0n = Real(0), x1n = Real(0), x2n = Real(0), an = Real(0);
        load_xa(rq[1], x0n, x1n, x2n, an);
        if (aq[0]) cp_wait_groups<D>();
        else fetch_sync(i, p % RING);

        Real tv[CPT];
        if constexpr (std::is_same<Real, float>::value) {
            // ---- local pass -------------------------------------------------
            float gmin = INF, gmax = -INF, s1 = 0.f, s2 = 0.f, rsum = 0.f;
            int jmin = jbase, jmax = 0x7FFFFFFF, nnz = 0;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float4 t4 = *reinterpret_cast<const float4 *>(slot + 4 * (tid + NT * g));
                float4 c4;
                if (!PTS) c4 = *reinterpret_cast<const float4 *>(slot + WID + 4 * (tid + NT * g));
                const float ts[4] = {t4.x, t4.y, t4.z, t4.w};
                const float cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = 4 * g + e, j = jbase + 4 * NT * g + e;
                    const float t = ts[e];
                    tv[c] = t;
                    const float cst = PTS ? cost3(x0c, x1c, x2c, y0[c], y1[c], y2[c]) : cs[e];
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
            }
            const uint32_t kmin = f2key(gmin);
            const uint32_t kmax = (jmax == 0x7FFFFFFF) ? 0u : f2key(gmax);
            Red<float> R = block_reduce<AWAY, NW>(red, par, sums, cnt, kmin, jmin, s1, s2, kmax, jmax, nnz, rsum);
            par ^= 1;
            if (!isfinite(R.gmin)) { if (tid == 0) atomicCAS(A.status, 0, (int)kDevNonFinite); break; }
            const float t_js = slot[R.jmin];
            const float t_v = (AWAY && R.jmax >= 0 && R.jmax < n) ? slot[R.jmax] : 0.f;
            const Step<float> S = decide<float>(R, ac, t_js, t_v, A.variant, A.step, rho, m, k);
            // ---- update ----------------------------------------------------
            float *trow = A.T + (size_t)i * n;
            if (S.kind == 2) {
                // pairwise: only j* and v change
                const float dv = S.drop ? -t_v : -S.sub_v;
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 4 * g + e, j = jbase + 4 * NT * g + e;
                        if (j == S.js && S.add_js != 0.f) {
                            const float tn = tv[c] + S.add_js;
                            kahan2(q[c], qc[c], rho * (tn - tv[c]));
                            trow[j] = tn;
                        }
                        if (j == S.v && dv != 0.f) {
                            const float tn = S.drop ? 0.f : tv[c] + dv;
                            kahan2(q[c], qc[c], rho * (tn - tv[c]));
                            trow[j] = tn;
                        }
                    }
            } else if (S.kind >= 0) {
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 4 * g + e, j = jbase + 4 * NT * g + e;
                        const float t = tv[c];
                        const float tn = apply<float>(S, j, t);
                        if (tn != t) {
                            kahan2(q[c], qc[c], rho * (tn - t));
                            trow[j] = tn;
                        }
                    }
            }
            if (tid == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = i;
                A.trace[4 * k + 1] = R.jmin;
                A.trace[4 * k + 2] = trace_vdir((AWAY && R.jmax >= 0 && R.jmax < n) ? R.jmax : -1, S.kind);
                A.trace[4 * k + 3] = __float_as_int((float)S.gamma);
            }
        } else {
            double gmin = 0.0, gmax = 0.0, s1 = 0.0, s2 = 0.0;
            int jmin = 0x7FFFFFFF, jmax = 0x7FFFFFFF, nnz = 0;
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = 4 * g + e, j = jbase + 4 * NT * g + e;
                    const double t = slot[j];
                    tv[c] = t;
                    const double cst = PTS ? cost3(x0c, x1c, x2c, y0[c], y1[c], y2[c]) : slot[WID + j];
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
            const double t_js = slot[R.jmin];
            const double t_v = (AWAY && R.jmax >= 0 && R.jmax < n) ? (double)slot[R.jmax] : 0.0;
            const Step<double> S = decide<double>(R, (double)ac, t_js, t_v, A.variant, A.step, (double)rho, m, k);
            if (S.kind >= 0) {
                double *trow = A.T + (size_t)i * n;
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 4 * g + e, j = jbase + 4 * NT * g + e;
                        const double t = tv[c];
                        const double tn = apply<double>(S, j, t);
                        if (j < n && tn != t) {
                            q[c] = dadd(q[c], dsub(tn, t));
                            trow[j] = tn;
                        }
                    }
            }
            if (tid == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = i;
                A.trace[4 * k + 1] = R.jmin;
                A.trace[4 * k + 2] = trace_vdir((AWAY && R.jmax >= 0 && R.jmax < n) ? R.jmax : -1, S.kind);
                A.trace[4 * k + 3] = __float_as_int((float)S.gamma);
            }
        }
        // advance the pipeline
        i_prev = i;
#pragma unroll
        for (int t = 0; t < D + 1; ++t) rq[t] = rq[t + 1];
        rq[D + 1] = r_far;
#pragma unroll
        for (int t = 0; t < D; ++t) aq[t] = aq[t + 1];
        x0c = x0n; x1c = x1n; x2c = x2n; ac = an;
    }
    cp_wait_all();
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = 4 * g + e, j = jbase + 4 * NT * g + e;
            if constexpr (F32) {
                if (j < n) A.q[j] = (double)q[c] - (double)qc[c];
            } else {
                if (j < n) A.q[j] = q[c];
            }
        }
}

template <typename Real, int NT, int G, bool PTS>
static size_t epoch_smem(int ring) {
    constexpr int SLOT = NT * 4 * G * (PTS ? 1 : 2);
    size_t red_bytes = std::is_same<Real, float>::value ? sizeof(RedF) * 2 * kMaxWarps
                                                        : sizeof(RedD) * 2 * kMaxWarps;
    return (size_t)ring * SLOT * sizeof(Real) + red_bytes;
}

template <typename Real, int NT, int G, bool PTS, bool AWAY, int RING>
static void launch_ring(const EpochArgs<Real> &A, cudaStream_t st) {
    size_t smem = epoch_smem<Real, NT, G, PTS>(RING);
    auto kern = k_epoch<Real, NT, G, PTS, AWAY, RING>;
    static bool attr_set = false;  // one attribute call per instantiation and process
    if (!attr_set) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
        attr_set = true;
    }
    kern<<<1, NT, smem, st>>>(A);
}

// Four ring slots (rows streamed two updates ahead) when they fit in shared
// memory, else three (one update ahead).
template <typename Real, int NT, int G, bool PTS, bool AWAY>
static void launch_cfg(const EpochArgs<Real> &A, cudaStream_t st) {
    if (epoch_smem<Real, NT, G, PTS>(4) <= (size_t)kSmemMax)
        launch_ring<Real, NT, G, PTS, AWAY, 4>(A, st);
    else
        launch_ring<Real, NT, G, PTS, AWAY, 3>(A, st);
}

template <typename Real, int NT, int G>
static void launch_shape(const EpochArgs<Real> &A, cudaStream_t st) {
    bool pts = A.in.cost_mode == kCostPts3;
    bool away = A.variant == SR_OT_BCAFW || A.variant == SR_OT_BCPFW;
    if (pts) {
        if (away) launch_cfg<Real, NT, G, true, true>(A, st);
        else launch_cfg<Real, NT, G, true, false>(A, st);
    } else {
        if (away) launch_cfg<Real, NT, G, false, true>(A, st);
        else launch_cfg<Real, NT, G, false, false>(A, st);
    }
}

int epoch_max_n(bool fp64) { return fp64 ? 256 * 8 : 512 * 16; }

template <>
bool launch_epoch<float>(const EpochArgs<float> &A, cudaStream_t st) {
    const int n = A.in.n;
    if (n <= 256 * 4) launch_shape<float, 256, 1>(A, st);
    else if (n <= 256 * 8) launch_shape<float, 256, 2>(A, st);
    else if (n <= 256 * 16) launch_shape<float, 256, 4>(A, st);
    else if (n <= 512 * 16) launch_shape<float, 512, 4>(A, st);
    else return false;
    return true;
}

template <>
bool launch_epoch<double>(const EpochArgs<double> &A, cudaStream_t st) {
    const int n = A.in.n;
    if (n <= 256 * 4) launch_shape<double, 256, 1>(A, st);
    else if (n <= 256 * 8) launch_shape<double, 256, 2>(A, st);
    else return false;
    return true;
}

}  // namespace srot
