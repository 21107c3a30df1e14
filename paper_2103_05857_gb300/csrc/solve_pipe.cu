// solve_pipe.cu -- one epoch of BCPFW (pairwise steps, Alg. A.3, exact line
// search eq. 10) on a single instance, with the work of consecutive block
// updates overlapped.
//
// A pairwise step of row i changes the plan, and so the residual r, in two
// columns only: the LMO vertex j* and the away vertex v. Everything the next
// update needs can therefore be prepared while the current one is applied,
// over the columns it leaves unchanged, and completed afterwards at the two
// changed columns:
//   LMO of row p+1:    min over j not in {j*_p, v_p} of C_ij + q_j (taken by
//                      the compute warps), then the two values at j*_p, v_p
//                      with the updated q;
//   away vertex of p+1: max over its atoms not in {j*_p, v_p}; if an atom is
//                      one of those two columns, recomputed in full after the
//                      update.
// Both merges use the order of the plain kernel (value, then column), so the
// decisions are exactly those of the two-phase kernel (solve_sparse.cu).
//
// Two control warps alternate: in phase p the owner warp (p even: first,
// p odd: second) decides and applies update p with the atoms of row p it
// already holds, while the other warp loads the atoms of row p+1 and takes
// their statistics; after one named barrier (compute warps and owner arrive)
// it completes the LMO and the away vertex, publishes {j*_{p+1}, v_{p+1}} and
// becomes the owner of update p+1. One full barrier per update.
//
// Layout (atom records, compensated residual pair, record / cost-row ring,
// row-info ring written by compute warp 1, overflow hand-off) as in
// solve_sparse.cu. A row whose record is being rewritten (it repeats the
// previous row, uniform order) is read from global memory after the apply.
#include <algorithm>
#include <limits>

#include "atoms.cuh"
#include "common.cuh"
#include "cpasync.cuh"
#include "internal.h"
#include "step.cuh"

namespace srot {

namespace {

constexpr int kSmemMax = 227 * 1024;

__device__ inline void named_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
__device__ inline void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

}  // namespace

template <int NTC, int G, bool PTS, int RING>
__global__ void __launch_bounds__(NTC + 2 * kWarp, 1) k_epoch_pipe(EpochArgs<float> A) {
    constexpr int NWC = NTC / kWarp;  // compute warps; warps NWC, NWC+1 are the control warps
    constexpr int NT = NTC + 2 * kWarp;
    constexpr int CPT = 4 * G;
    constexpr int WID = NTC * CPT;
    constexpr int D = RING - 2;
    static_assert(D >= 1, "ring too small");
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
    SpRed *red = reinterpret_cast<SpRed *>(aring + RING * kAtomRecord);
    int *sflag = reinterpret_cast<int *>(red + NWC);      // [2..3]: exclusion set
    float4 *rinf = reinterpret_cast<float4 *>(sflag + 4);  // [2 * RING] row info

    const int m = A.in.m, n = A.in.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cw = warp - NWC;  // 0 / 1 for the control warps
    const bool ctrl = cw >= 0;
    const unsigned FULL = 0xffffffffu;
    const float rho = (float)A.rho;
    const int order = A.order;
    const bool vec = A.vec;
    int4 *grec = A.atoms;
    const float INF = std::numeric_limits<float>::infinity();

    // ---- one-time set-up ------------------------------------------------
    for (int j = tid; j < WID; j += NT) {
        if (j < n) {
            const double qq = A.q[j];
            const float h = (float)qq;
            qh[j] = h;
            ql[j] = (float)((double)h - qq);
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
        sflag[2] = -1;
        sflag[3] = -1;
        if (A.resume) *A.resume = -1;
    }
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
    // compute warp 0 streams atom records; all compute threads their cost quads
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
    float cst[CPT];
    auto load_costs = [&](int s, float x0, float x1, float x2) {
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
    // compute warp 1, lane 0: the row of the update in slot s and its data
    auto put_info = [&](int s, int i, bool pre, float x0, float x1, float x2, float ai) {
        const float ra = ai > 0.f ? 1.f / ai : 0.f;
        const float ia = ai > 0.f ? 1.f / (2.f * rho * ai) : 0.f;
        rinf[2 * s] = make_float4(__int_as_float(i), __int_as_float(pre ? 1 : 0), x0, x1);
        rinf[2 * s + 1] = make_float4(x2, ai, ra, ia);
    };
    // compute warps: partial argmin of the current cost row over the columns
    // not in {e1, e2}; ties to the smallest column
    auto partial_argmin = [&](int e1, int e2) {
        const int q1 = e1 >= 0 ? (e1 >> 2) : -1, q2 = e2 >= 0 ? (e2 >> 2) : -1;
        float qv[G];
        int qj[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int qi = tid + NTC * g;
            const int j0 = 4 * qi;
            const float4 q4 = *reinterpret_cast<const float4 *>(qh + j0);
            float2 ga = __fadd2_rn(make_float2(cst[4 * g], cst[4 * g + 1]), make_float2(q4.x, q4.y));
            float2 gb = __fadd2_rn(make_float2(cst[4 * g + 2], cst[4 * g + 3]), make_float2(q4.z, q4.w));
            if (qi == q1 || qi == q2) {  // an excluded column in this quad
                const int mk = (qi == q1 ? 1 << (e1 & 3) : 0) | (qi == q2 ? 1 << (e2 & 3) : 0);
                if (mk & 1) ga.x = INF;
                if (mk & 2) ga.y = INF;
                if (mk & 4) gb.x = INF;
                if (mk & 8) gb.y = INF;
            }
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
        const uint32_t km = f2key(qv[0]);
        const uint32_t wk = __reduce_min_sync(FULL, km);
        const int wj = __reduce_min_sync(FULL, km == wk ? qj[0] : 0x7FFFFFFF);
        if (lane == 0) red[warp] = SpRed{wk, wj};
    };
    // control warps: gradient of a row (x, cost slot s) at column j, current residual
    auto grad_at = [&](int j, int s, float x0, float x1, float x2) -> float {
        float c;
        if (PTS) {
            const float4 y = ys[j];
            const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
            c = fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0)));
        } else {
            c = cring[(size_t)s * WID + j];
        }
        return c + qh[j];
    };

    const bool prefetchable = (order == SR_OT_CYCLIC || order == SR_OT_PERMUTE || order == SR_OT_UNIFORM);
    // Compute threads: rq[t] = row of update p+1+t (t <= D), aq[t]: it travels
    // by cp.async. Row p+1+D is issued in phase p into slot (p+1+D) % RING; a
    // row whose record changes between its fetch and its use is not issued.
    int rq[D + 1];
    bool aq[D + 1];
    int row_cur = row_of(0), row_prev = -1;
    // compute threads: x, a of the row whose cost row they build next (loaded
    // one phase before use, so no global-load latency sits in a phase)
    float xn0 = 0.f, xn1 = 0.f, xn2 = 0.f, an = 0.f;
    if (!ctrl) {
        int pre[D + 1];
#pragma unroll
        for (int t = 0; t <= D; ++t) {
            pre[t] = row_of(t);
            bool ok = prefetchable && pre[t] >= 0;
#pragma unroll
            for (int u = 0; u < t; ++u) ok = ok && pre[t] != pre[u];
            if (ok) fetch_async(pre[t], t % RING);
            commit();
            if (t >= 1) { rq[t - 1] = pre[t]; aq[t - 1] = ok; }
        }
        rq[D] = row_of(D + 1);
        aq[D] = false;
        const bool ok0 = prefetchable && pre[0] >= 0;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, a0 = 0.f;
        load_x(pre[0], x0, x1, x2, a0);
        if (ok0) wait_groups<D>();  // row 0: record (warp 0) and costs
        else if (!PTS) fetch_sync_costs(pre[0], 0);
        if (warp == 1 && lane == 0) put_info(0, pre[0], ok0, x0, x1, x2, a0);
        load_x(rq[0], xn0, xn1, xn2, an);
        load_costs(0, x0, x1, x2);  // PTS: from x; given C: slot 0 (own quads)
    }
    __syncthreads();  // row 0's record, costs and info visible

    // control-warp state of the update this warp owns next
    LaneAtoms at;
    AtomStats st;
    DF tvd{0.f, 0.f};
    float gmin = 0.f, gmx = 0.f, inv = 0.f, ai = 0.f;
    int js = 0, row = 0;
    int stop_l = 0;

    // the statistics warp for row `pr` (slot s): atoms, away vertex over the
    // atoms not in {e1, e2}, then (after the named barrier) the LMO merge and
    // the completion at e1, e2; publishes the exclusion set of update pr
    auto stats_and_merge = [&](int s, int e1, int e2, bool arrive_before) {
        const float4 r0 = rinf[2 * s], r1 = rinf[2 * s + 1];
        const int i1 = __float_as_int(r0.x);
        const bool pre1 = __float_as_int(r0.y) != 0;
        const float x0 = r0.z, x1 = r0.w, x2 = r1.x, a1 = r1.y, ra = r1.z, ia = r1.w;
        bool full_after = !pre1;  // record read (and statistics) after the update
        bool anyE = false;
        if (pre1) {
            at = load_atoms(aring + (size_t)s * kAtomRecord, lane);
            const bool e_in = (at.j[0] >= 0 && (at.j[0] == e1 || at.j[0] == e2)) ||
                              (at.j[1] >= 0 && (at.j[1] == e1 || at.j[1] == e2));
            anyE = __any_sync(FULL, e_in);
            if (!anyE) {
                auto grad = [&](int j) -> float { return grad_at(j, s, x0, x1, x2); };
                st = atom_stats(at, grad, a1, false, &tvd);
            }
        }
        if (arrive_before) named_sync(1, NT);
        if (full_after) {
            fetch_sync_record(i1, s);
            __syncwarp();
            at = load_atoms(aring + (size_t)s * kAtomRecord, lane);
        }
        if (full_after || anyE) {
            auto grad = [&](int j) -> float { return grad_at(j, s, x0, x1, x2); };
            st = atom_stats(at, grad, a1, false, &tvd);
        }
        // LMO: the compute warps' partial minimum and the columns e1, e2
        const SpRed e = lane < NWC ? red[lane] : SpRed{0xFFFFFFFFu, 0x7FFFFFFF};
        uint32_t wk = e.kmin;
        int wj = e.jmin;
        const int ec = lane == NWC ? e1 : (lane == NWC + 1 ? e2 : -1);
        if (ec >= 0) {
            wk = f2key(grad_at(ec, s, x0, x1, x2));
            wj = ec;
        }
        const uint32_t fk = __reduce_min_sync(FULL, wk);
        js = __reduce_min_sync(FULL, wk == fk ? wj : 0x7FFFFFFF);
        gmin = key2f(fk);
        row = i1;
        ai = a1;
        gmx = inv = 0.f;
        if (a1 > 0.f) {
            gmx = st.t_v * ra;  // same rounding as the two-phase kernel
            inv = ia;
        }
        if (!isfinite(gmin)) {
            if (lane == 0) atomicCAS(A.status, 0, (int)kDevNonFinite);
            stop_l = 1;
        }
        if (lane == 0) {
            sflag[2] = js;
            sflag[3] = (st.v >= 0 && st.v < n) ? st.v : -1;
        }
    };

    // ---- prologue phase: LMO and away vertex of row 0 ---------------------
    if (!ctrl) {
        partial_argmin(-1, -1);
        named_arrive(1, NT);
        if (m > 1) {
            if (aq[0]) wait_groups<D - 1>();  // row 1: record and costs
            else if (!PTS) fetch_sync_costs(rq[0], 1 % RING);
            load_costs(1 % RING, xn0, xn1, xn2);
            if (warp == 1 && lane == 0) put_info(1 % RING, rq[0], aq[0], xn0, xn1, xn2, an);
            load_x(row_of(2), xn0, xn1, xn2, an);  // row 2, used in phase 0
        }
    } else if (cw == 0) {
        stats_and_merge(0, -1, -1, true);
    } else {
        named_arrive(1, NT);
    }
    if (__syncthreads_or(stop_l)) {
        wait_groups<0>();
        __syncthreads();
        for (int j = tid; j < n; j += NT) A.q[j] = (double)qh[j] - (double)ql[j];
        return;
    }

    for (int p = 0; p < m; ++p) {
        const long long k = A.k0 + p;
        const bool more = p + 1 < m;
        const int e1 = sflag[2], e2 = sflag[3];  // columns update p changes
        if (!ctrl) {
            // issue row p+1+D (not if its record changes before it is used)
            const int rnew = row_of(p + 1 + D);
            bool ok = prefetchable && rnew >= 0 && rnew != row_cur && rnew != row_prev;
#pragma unroll
            for (int u = 0; u < D; ++u) ok = ok && rnew != rq[u];
            if (ok) fetch_async(rnew, (p + 1 + D) % RING);
            rq[D] = rnew;
            aq[D] = ok;
        }
        commit();
        if (!ctrl) {
            if (more) {
                partial_argmin(e1, e2);  // row p+1
                named_arrive(1, NT);
                if (p + 2 < m) {
                    if (aq[1]) wait_groups<D - 1>();  // row p+2: record and costs
                    else if (!PTS) fetch_sync_costs(rq[1], (p + 2) % RING);
                    load_costs((p + 2) % RING, xn0, xn1, xn2);  // x of row p+2, loaded last phase
                    if (warp == 1 && lane == 0) put_info((p + 2) % RING, rq[1], aq[1], xn0, xn1, xn2, an);
                    load_x(row_of(p + 3), xn0, xn1, xn2, an);    // for the next phase
                }
            }
        } else if (cw == (p & 1)) {
            // ---- owner: update p ------------------------------------------
            bool present = false;
            int jpos = -1;
            atom_weight(at, js, &present, &jpos);
            const Step<float> S = decide_pairwise(st, gmin, js, ai, rho, gmx, inv, n);
            const bool ok = apply_pairwise(S, at, jpos, st.vpos, tvd, rho, A.T + (size_t)row * n, qh, ql,
                                           grec + (size_t)row * kAtomRecord, lane);
            if (lane == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = row;
                A.trace[4 * k + 1] = js;
                A.trace[4 * k + 2] = trace_vdir((st.v >= 0 && st.v < n) ? st.v : -1, S.kind);
                A.trace[4 * k + 3] = __float_as_int(S.gamma);
            }
            if (!ok) {
                stop_l = 1;  // j* would be a 64th atom: the dense kernel takes over at p
                if (lane == 0 && A.resume) *A.resume = p;
                if (lane == 0 && A.sticky) *A.sticky = 1;
            }
            if (more) named_arrive(1, NT);
        } else if (more) {
            // ---- statistics warp: row p+1 ---------------------------------
            stats_and_merge((p + 1) % RING, e1, e2, true);
        }
        if (__syncthreads_or(stop_l)) break;
        if (!ctrl) {
            row_prev = row_cur;
            row_cur = rq[0];
#pragma unroll
            for (int t = 0; t < D; ++t) { rq[t] = rq[t + 1]; aq[t] = aq[t + 1]; }
        }
    }
    wait_groups<0>();
    __syncthreads();
    for (int j = tid; j < n; j += NT) A.q[j] = (double)qh[j] - (double)ql[j];
}

template <int NT, int G, bool PTS>
static size_t pipe_smem(int ring) {
    constexpr int WID = NT * 4 * G;
    size_t b = 2 * (size_t)WID * 4;
    if (PTS) b += (size_t)WID * 16;
    else b += (size_t)ring * WID * 4;
    b += (size_t)ring * kAtomRecord * 16;
    b += (NT / kWarp) * sizeof(SpRed) + 16;
    b += (size_t)ring * 32;  // row-info ring
    return b;
}

template <int NT, int G, bool PTS, int RING>
static void launch_pipe_ring(const EpochArgs<float> &A, cudaStream_t st) {
    auto kern = k_epoch_pipe<NT, G, PTS, RING>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
        attr_set = true;
    }
    kern<<<1, NT + 2 * kWarp, pipe_smem<NT, G, PTS>(RING), st>>>(A);
}

template <int NT, int G>
static void launch_pipe(const EpochArgs<float> &A, cudaStream_t st) {
    if (A.in.cost_mode == kCostPts3) {
        launch_pipe_ring<NT, G, true, 4>(A, st);
    } else {
        if (pipe_smem<NT, G, false>(4) <= (size_t)kSmemMax) launch_pipe_ring<NT, G, false, 4>(A, st);
        else launch_pipe_ring<NT, G, false, 3>(A, st);
    }
}

bool launch_epoch_pipe(const EpochArgs<float> &A, cudaStream_t st) {
    if (A.variant != SR_OT_BCPFW) return false;
    const int n = A.in.n;
    if (n <= 256 * 4) launch_pipe<256, 1>(A, st);
    else if (n <= 256 * 8) launch_pipe<256, 2>(A, st);
    else if (n <= 256 * 16) launch_pipe<256, 4>(A, st);
    else if (n <= 512 * 16) launch_pipe<512, 4>(A, st);
    else return false;
    return true;
}

}  // namespace srot
