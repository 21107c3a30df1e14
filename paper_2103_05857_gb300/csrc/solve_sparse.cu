// solve_sparse.cu -- one epoch of BCPFW / BCAFW (FP32) with per-row active
// sets kept as compact atom lists.
//
// With away or pairwise steps (Sec. 4.1, Alg. A.2, A.3) a row's active set
// S_i = {j : t_ij > 0} stays small, and the paper notes that these steps cost
// O(n + |S_i|) per block (Sec. 4.3). This kernel follows that count: per
// block update the only O(n) work is the LMO argmin of the row gradient
// (eq. 7); the away vertex, the line search (eq. 10) and the rank-1 update
// touch the |S_i| atoms only.
//
// Layout. One CTA of NT threads. Thread tid owns columns j = 4 (tid + NT g)+e
// as in the dense kernel; the target points y_j of those columns live in
// registers as pairs for packed FP32x2 arithmetic. The running residual
// q = rho (T^T 1 - b) lives in shared memory as a compensated FP32 pair
// (qh, ql), initialised from the exact FP64 column sums and updated only at
// the columns an update changes, so its value never drifts by the FP32
// rounding of large partial sums. Each row's atoms are a 1 KiB record
// {count, (j, t) x 63} with double-float weights (so steps conserve the row's
// mass) in global memory, streamed into a shared-memory ring RING-2 updates
// ahead (cp.async) by a control warp, which alone applies the update. The
// dense plan T is kept exact by storing the changed entries.
//
// Per update: argmin pass (compute warps) | away vertex (control warp) ->
// barrier -> control warp: global argmin, decision, atom / T / q updates |
// compute warps: next cost row -> barrier. (For pairwise steps the
// pipelined kernel of solve_pipe.cu is the default; this one is kept for
// away steps and as its reference.)
//
// If a row would need more than 63 atoms, the kernel stops before changing
// it and records the update index in *resume; the dense kernel then finishes
// the epoch from there and the solve continues on the dense path.
#include <limits>

#include <algorithm>

#include "atoms.cuh"
#include "common.cuh"
#include "cpasync.cuh"
#include "internal.h"
#include "step.cuh"

namespace srot {

namespace {

constexpr int kSmemMax = 227 * 1024;

}  // namespace

template <int NTC, int G, bool PTS, int RING, bool PAIR>
__global__ void __launch_bounds__(NTC + kWarp, 1) k_epoch_sparse(EpochArgs<float> A) {
    constexpr int NWC = NTC / kWarp;  // compute warps; warp NWC is the control warp
    constexpr int NT = NTC + kWarp;
    constexpr int CPT = 4 * G;
    constexpr int WID = NTC * CPT;
    constexpr int D = RING - 2;
    // a row outgrew its atom record in an earlier epoch: the dense kernel
    // takes every epoch from now on (its records are no longer kept)
    if (A.sticky && *reinterpret_cast<const volatile int *>(A.sticky)) {
        if (threadIdx.x == 0 && A.resume) *A.resume = 0;
        return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    float *qh = reinterpret_cast<float *>(smem);
    float *ql = qh + WID;
    float4 *ys = reinterpret_cast<float4 *>(ql + WID);
    float *cring = reinterpret_cast<float *>(ys + (PTS ? WID : 0));
    int4 *aring = reinterpret_cast<int4 *>(cring + (PTS ? 0 : RING * WID));
    SpRed(*red)[NWC] = reinterpret_cast<SpRed(*)[NWC]>(aring + RING * kAtomRecord);
    int *sflag = reinterpret_cast<int *>(red + 2);
    // per ring slot, the row of that update and what the control warp needs of
    // it, written one update ahead by compute warp 1 (off the control chain)
    float4 *rinf = reinterpret_cast<float4 *>(sflag + 4);  // [2 * RING]

    const int m = A.in.m, n = A.in.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool ctrl = warp == NWC;
    const unsigned FULL = 0xffffffffu;
    const float rho = (float)A.rho;
    const int order = A.order;
    const bool vec = A.vec;
    int4 *grec = A.atoms;

    // ---- one-time set-up: residual pair, point table, padding ------------
    for (int j = tid; j < WID; j += NT) {
        if (j < n) {
            const double qq = A.q[j];
            const float h = (float)qq;
            qh[j] = h;
            ql[j] = (float)((double)h - qq);  // value = qh - ql
        } else {
            qh[j] = 1e30f;
            ql[j] = 0.f;
        }
        if (PTS)
            ys[j] = j < n ? make_float4(A.in.Y[(size_t)j * 3], A.in.Y[(size_t)j * 3 + 1],
                                        A.in.Y[(size_t)j * 3 + 2], 0.f)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
        if (!PTS)
            for (int s = 0; s < RING; ++s) cring[(size_t)s * WID + j] = 0.f;
    }
    if (tid == 0) {
        sflag[0] = 0;
        if (A.resume) *A.resume = -1;
    }
    // compute threads: negated target points of their columns, in pairs
    float2 ny0[PTS ? 2 * G : 1], ny1[PTS ? 2 * G : 1], ny2[PTS ? 2 * G : 1];
    if (PTS && !ctrl) {
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 4 * (tid + NTC * g) + 2 * h;
                const bool a0 = j < n, a1 = j + 1 < n;
                ny0[2 * g + h] = make_float2(a0 ? -A.in.Y[(size_t)j * 3] : 0.f, a1 ? -A.in.Y[(size_t)(j + 1) * 3] : 0.f);
                ny1[2 * g + h] = make_float2(a0 ? -A.in.Y[(size_t)j * 3 + 1] : 0.f, a1 ? -A.in.Y[(size_t)(j + 1) * 3 + 1] : 0.f);
                ny2[2 * g + h] = make_float2(a0 ? -A.in.Y[(size_t)j * 3 + 2] : 0.f, a1 ? -A.in.Y[(size_t)(j + 1) * 3 + 2] : 0.f);
            }
    }
    __syncthreads();

    auto row_of = [&](int p) -> int {
        if (p >= m) return -1;
        if (order == SR_OT_CYCLIC) return p;
        if (order == SR_OT_PERMUTE) return A.perm[p];
        return scale_u64(sm64_draw(A.seed, 2, (uint64_t)(A.k0 + p)), m);
    };
    // control warp: atom record; compute threads: their quads of the cost row
    // compute warp 0 streams the atom records (off the control warp's chain);
    // it waits for them before the barrier that precedes their use
    auto fetch_async = [&](int i, int s) {
        if (warp == 0) {
            cp16(aring + (size_t)s * kAtomRecord + lane, grec + (size_t)i * kAtomRecord + lane);
            cp16(aring + (size_t)s * kAtomRecord + 32 + lane, grec + (size_t)i * kAtomRecord + 32 + lane);
        }
        if (!ctrl && !PTS) {
            float *dst = cring + (size_t)s * WID;
            const float *src = A.in.C + (size_t)i * n;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j0 = 4 * (tid + NTC * g);
                if (vec && j0 + 3 < n) cp16(dst + j0, src + j0);
                else
                    for (int e = 0; e < 4; ++e)
                        if (j0 + e < n) cp4(dst + j0 + e, src + j0 + e);
            }
        }
    };
    auto fetch_sync_record = [&](int i, int s) {
        aring[(size_t)s * kAtomRecord + lane] = grec[(size_t)i * kAtomRecord + lane];
        aring[(size_t)s * kAtomRecord + 32 + lane] = grec[(size_t)i * kAtomRecord + 32 + lane];
    };
    auto fetch_sync_costs = [&](int i, int s) {
        float *dst = cring + (size_t)s * WID;
        const float *src = A.in.C + (size_t)i * n;
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * (tid + NTC * g) + e;
                if (j < n) dst[j] = src[j];
            }
    };
    // compute threads: the cost of their columns for row i (slot s when given)
    float cst[CPT];
    auto load_costs = [&](int i, int s, float x0, float x1, float x2) {
        if (i < 0) return;
        if (PTS) {
            const float2 X0 = make_float2(x0, x0), X1 = make_float2(x1, x1), X2 = make_float2(x2, x2);
#pragma unroll
            for (int h = 0; h < 2 * G; ++h) {
                const float2 d0 = __fadd2_rn(X0, ny0[h]), d1 = __fadd2_rn(X1, ny1[h]), d2 = __fadd2_rn(X2, ny2[h]);
                float2 c = __fmul2_rn(d0, d0);
                c = __ffma2_rn(d1, d1, c);
                c = __ffma2_rn(d2, d2, c);
                cst[2 * h] = c.x;
                cst[2 * h + 1] = c.y;
            }
        } else {
            const float *cs = cring + (size_t)s * WID;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float4 c4 = *reinterpret_cast<const float4 *>(cs + 4 * (tid + NTC * g));
                cst[4 * g] = c4.x;
                cst[4 * g + 1] = c4.y;
                cst[4 * g + 2] = c4.z;
                cst[4 * g + 3] = c4.w;
            }
        }
    };
    auto load_x = [&](int i, float &x0, float &x1, float &x2, float &ai) {
        if (i < 0) return;
        if (PTS) {
            x0 = A.in.X[(size_t)i * 3];
            x1 = A.in.X[(size_t)i * 3 + 1];
            x2 = A.in.X[(size_t)i * 3 + 2];
        }
        ai = A.in.a[i];
    };
    // pairwise steps: 1 / a_i and 1 / (2 rho a_i), taken two updates ahead
    auto recips = [&](float ai, float &ra, float &ia) {
        ra = ai > 0.f ? 1.f / ai : 0.f;
        ia = ai > 0.f ? 1.f / (2.f * rho * ai) : 0.f;
    };
    // compute warp 1, lane 0: row info of the update in ring slot s
    auto put_info = [&](int s, int i, bool pre, float x0, float x1, float x2, float ai) {
        float ra = 0.f, ia = 0.f;
        if (PAIR) recips(ai, ra, ia);
        rinf[2 * s] = make_float4(__int_as_float(i), __int_as_float(pre ? 1 : 0), x0, x1);
        rinf[2 * s + 1] = make_float4(x2, ai, ra, ia);
    };

    const bool prefetchable = (order == SR_OT_CYCLIC || order == SR_OT_PERMUTE || order == SR_OT_UNIFORM);
    // Pipelines: rq[t] = row of update p+t (t <= D+1), aq[t] = it travels by
    // cp.async (t < D); x, a of the rows of updates p, p+1 (c, n).
    int rq[D + 2];
    bool aq[D + 1];
#pragma unroll
    for (int t = 0; t < D + 2; ++t) rq[t] = row_of(t);
#pragma unroll
    for (int t = 0; t < D; ++t) {
        bool ok = prefetchable && rq[t] >= 0;
#pragma unroll
        for (int u = 0; u < t; ++u) ok = ok && rq[t] != rq[u];
        aq[t] = ok;
        if (ok) fetch_async(rq[t], t % RING);
        commit();
    }
    float xc0 = 0.f, xc1 = 0.f, xc2 = 0.f, ac = 0.f, xn0 = 0.f, xn1 = 0.f, xn2 = 0.f, an = 0.f;
    load_x(rq[0], xc0, xc1, xc2, ac);
    load_x(rq[1], xn0, xn1, xn2, an);
    if (warp == 1 && lane == 0) put_info(0, rq[0], aq[0], xc0, xc1, xc2, ac);
    if (!ctrl) {
        if (!PTS) {
            if (aq[0]) wait_groups<D - 1>();
            else fetch_sync_costs(rq[0], 0);
        } else if (warp == 0 && aq[0]) {
            wait_groups<D - 1>();  // the record of row 0
        }
        load_costs(rq[0], 0, xc0, xc1, xc2);
    }
    __syncthreads();  // records streamed by warp 0 visible to the control warp
    int i_prev = -1, par = 0;
    int stop_l = 0;  // control warp: stop after this update
    for (int p = 0; p < m; ++p) {
        const long long k = A.k0 + p;
        const int s_cur = p % RING;
        int i, r_far = -1;
        float xm0 = 0.f, xm1 = 0.f, xm2 = 0.f, am = 0.f;  // row of update p+2
        float rc = 0.f, ic = 0.f;
        bool pre = false;
        if (ctrl) {
            // the row of this update and its data, from the row-info ring
            const float4 r0 = rinf[2 * s_cur], r1 = rinf[2 * s_cur + 1];
            i = __float_as_int(r0.x);
            pre = __float_as_int(r0.y) != 0;
            xc0 = r0.z; xc1 = r0.w; xc2 = r1.x; ac = r1.y; rc = r1.z; ic = r1.w;
        } else {
            i = rq[0];
            bool ok = prefetchable && rq[D] >= 0 && rq[D] != i_prev;
#pragma unroll
            for (int u = 0; u < D; ++u) ok = ok && rq[D] != rq[u];
            aq[D] = ok;
            if (ok) fetch_async(rq[D], (p + D) % RING);
            r_far = row_of(p + D + 2);
            load_x(rq[2 <= D + 1 ? 2 : D + 1], xm0, xm1, xm2, am);
        }
        commit();

        // ---- phase 1: LMO argmin (compute warps) | away vertex (control) ---
        LaneAtoms at;
        AtomStats st;
        DF t_vdf{0.f, 0.f};
        float gmx = 0.f, inv = 0.f;
        if (!ctrl) {
            // per quad a two-level tree, then across quads; on equal values the
            // lower column wins, so ties go to the smallest j overall
            float qv[G];
            int qj[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j0 = 4 * (tid + NTC * g);
                const float4 q4 = *reinterpret_cast<const float4 *>(qh + j0);
                const float2 ga = __fadd2_rn(make_float2(cst[4 * g], cst[4 * g + 1]), make_float2(q4.x, q4.y));
                const float2 gb = __fadd2_rn(make_float2(cst[4 * g + 2], cst[4 * g + 3]), make_float2(q4.z, q4.w));
                const bool ta = ga.y < ga.x, tb = gb.y < gb.x;
                const float va = ta ? ga.y : ga.x, vb = tb ? gb.y : gb.x;
                const int ia = j0 + (ta ? 1 : 0), ib = j0 + (tb ? 3 : 2);
                const bool tq = vb < va;
                qv[g] = tq ? vb : va;
                qj[g] = tq ? ib : ia;
            }
#pragma unroll
            for (int w = 1; w < G; w <<= 1)
#pragma unroll
                for (int g = 0; g + w < G; g += 2 * w)
                    if (qv[g + w] < qv[g]) { qv[g] = qv[g + w]; qj[g] = qj[g + w]; }
            const float gmin = qv[0];
            const int jmin = qj[0];
            const uint32_t km = f2key(gmin);
            const uint32_t wk = __reduce_min_sync(FULL, km);
            const int wj = __reduce_min_sync(FULL, km == wk ? jmin : 0x7FFFFFFF);
            if (lane == 0) red[par][warp] = SpRed{wk, wj};
        } else {
            if (!pre) {
                fetch_sync_record(i, s_cur);
                __syncwarp();
            }
            at = load_atoms(aring + (size_t)s_cur * kAtomRecord, lane);
            auto grad = [&](int j) -> float {
                float c;
                if (PTS) {
                    const float4 y = ys[j];
                    const float d0 = xc0 - y.x, d1 = xc1 - y.y, d2 = xc2 - y.z;
                    c = fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0)));
                } else {
                    c = __ldg(A.in.C + (size_t)i * n + j);
                }
                return c + qh[j];
            };
            st = atom_stats(at, grad, ac, !PAIR, &t_vdf);
            // quantities of the pairwise step that do not depend on the LMO vertex
            if (PAIR && ac > 0.f) {
                gmx = st.t_v * rc;  // gamma_max = alpha_v = t_v / a_i
                inv = ic;           // eq. 10 with d = a_i (e_j* - e_v)
            }
        }
        __syncthreads();  // (A)

        // ---- phase 2: decision and update (control) | next costs (compute) -
        if (ctrl) {
            const SpRed e = lane < NWC ? red[par][lane] : SpRed{0xFFFFFFFFu, 0x7FFFFFFF};
            const uint32_t wk = __reduce_min_sync(FULL, e.kmin);
            const int js = __reduce_min_sync(FULL, e.kmin == wk ? e.jmin : 0x7FFFFFFF);
            const float gmin_all = key2f(wk);
            bool present = false;
            int jpos = -1;
            const float t_js = atom_weight(at, js, &present, &jpos);
            bool stop = false;
            if (!isfinite(gmin_all)) {
                if (lane == 0) atomicCAS(A.status, 0, (int)kDevNonFinite);
                stop = true;
                stop_l = 1;
            }
            Step<float> S{-1, 0.f, js, st.v, 1.f, 0.f, 0.f, false};
            if (!stop)
                S = PAIR ? decide_pairwise(st, gmin_all, js, ac, rho, gmx, inv, n)
                         : decide_atoms(st, gmin_all, js, t_js, ac, A.variant, A.step, rho, m, k);
            const bool applied =
                stop || (PAIR ? apply_pairwise(S, at, jpos, st.vpos, t_vdf, rho, A.T + (size_t)i * n, qh, ql,
                                               grec + (size_t)i * kAtomRecord, lane)
                              : apply_atoms(S, at, present, t_vdf, ac, rho, A.T + (size_t)i * n, qh, ql,
                                            grec + (size_t)i * kAtomRecord, lane));
            if (!applied) {
                stop_l = 1;  // j* would be a 64th atom: the dense kernel takes over here
                if (lane == 0 && A.resume) *A.resume = p;
                if (lane == 0 && A.sticky) *A.sticky = 1;
            }
            if (lane == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = i;
                A.trace[4 * k + 1] = js;
                A.trace[4 * k + 2] = trace_vdir((st.v >= 0 && st.v < n) ? st.v : -1, S.kind);
                A.trace[4 * k + 3] = __float_as_int(S.gamma);
            }
        } else if (p + 1 < m) {
            if (!PTS) {
                if (aq[1]) wait_groups<D - 1>();
                else fetch_sync_costs(rq[1], (p + 1) % RING);
            } else if (warp == 0 && aq[1]) {
                wait_groups<D - 1>();  // the record of the next row
            }
            load_costs(rq[1], (p + 1) % RING, xn0, xn1, xn2);
            if (warp == 1 && lane == 0) put_info((p + 1) % RING, rq[1], aq[1], xn0, xn1, xn2, an);
        }
        par ^= 1;
        // (B) residual, records and next costs ready; stop if the control warp says so
        if (__syncthreads_or(stop_l)) break;
        if (!ctrl) {
            i_prev = i;
#pragma unroll
            for (int t = 0; t < D + 1; ++t) rq[t] = rq[t + 1];
            rq[D + 1] = r_far;
#pragma unroll
            for (int t = 0; t < D; ++t) aq[t] = aq[t + 1];
            xc0 = xn0; xc1 = xn1; xc2 = xn2; ac = an;
            xn0 = xm0; xn1 = xm1; xn2 = xm2; an = am;
        }
    }
    wait_groups<0>();
    __syncthreads();
    for (int j = tid; j < n; j += NT) A.q[j] = (double)qh[j] - (double)ql[j];
}

template <int NT, int G, bool PTS>
static size_t sparse_smem(int ring) {
    constexpr int WID = NT * 4 * G;  // NT: compute threads
    size_t b = 2 * (size_t)WID * 4;             // qh, ql
    if (PTS) b += (size_t)WID * 16;             // y table
    else b += (size_t)ring * WID * 4;           // cost-row ring
    b += (size_t)ring * kAtomRecord * 16;       // atom-record ring (1 KiB per slot)
    b += 2 * (NT / kWarp) * sizeof(SpRed) + 16; // reduction slots, flag
    b += (size_t)ring * 32;                     // row-info ring
    return b;
}

template <int NT, int G, bool PTS, int RING, bool PAIR>
static void launch_sp_ring(const EpochArgs<float> &A, cudaStream_t st) {
    auto kern = k_epoch_sparse<NT, G, PTS, RING, PAIR>;
    static bool attr_set = false;  // one attribute call per instantiation and process
    if (!attr_set) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
        attr_set = true;
    }
    kern<<<1, NT + kWarp, sparse_smem<NT, G, PTS>(RING), st>>>(A);
}

template <int NT, int G, bool PAIR>
static void launch_sp_var(const EpochArgs<float> &A, cudaStream_t st) {
    if (A.in.cost_mode == kCostPts3) {
        launch_sp_ring<NT, G, true, 4, PAIR>(A, st);
    } else {
        if (sparse_smem<NT, G, false>(4) <= (size_t)kSmemMax) launch_sp_ring<NT, G, false, 4, PAIR>(A, st);
        else launch_sp_ring<NT, G, false, 3, PAIR>(A, st);
    }
}

template <int NT, int G>
static void launch_sp(const EpochArgs<float> &A, cudaStream_t st) {
    if (A.variant == SR_OT_BCPFW) launch_sp_var<NT, G, true>(A, st);
    else launch_sp_var<NT, G, false>(A, st);
}

bool launch_epoch_sparse(const EpochArgs<float> &A, cudaStream_t st) {
    const int n = A.in.n;
    if (n <= 256 * 4) launch_sp<256, 1>(A, st);
    else if (n <= 256 * 8) launch_sp<256, 2>(A, st);
    else if (n <= 256 * 16) launch_sp<256, 4>(A, st);
    else if (n <= 512 * 16) launch_sp<512, 4>(A, st);
    else return false;
    return true;
}

// ---------------------------------------------------------------------------
// Atom records from a dense plan: one warp per row. *overflow is set when a
// row has more than 63 positive entries.
// ---------------------------------------------------------------------------
__global__ void k_build_atoms(int m, int n, const float *__restrict__ T, int4 *__restrict__ rec,
                              int *__restrict__ overflow) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    constexpr int K = kAtomRecord - 1;
    for (int i = w; i < m; i += nw) {
        const float *ti = T + (size_t)i * n;
        int4 *g = rec + (size_t)i * kAtomRecord;
        int cnt = 0;
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const float t = j < n ? ti[j] : 0.f;
            const bool act = t > 0.f;
            const unsigned mk = __ballot_sync(0xffffffffu, act);
            const int pos = cnt + __popc(mk & ((1u << lane) - 1u));
            if (act && pos < K) g[1 + pos] = make_int4(j, __float_as_int(t), 0, 0);
            cnt += __popc(mk);
        }
        if (lane == 0) {
            g[0] = make_int4(cnt < K ? cnt : K, 0, 0, 0);
            if (cnt > K) atomicExch(overflow, 1);
        }
    }
}

void launch_build_atoms(int m, int n, const float *T, int4 *rec, int *overflow, cudaStream_t st) {
    int blocks = std::min((m + 7) / 8, 152 * 4);
    k_build_atoms<<<blocks, 256, 0, st>>>(m, n, T, rec, overflow);
}

}  // namespace srot
