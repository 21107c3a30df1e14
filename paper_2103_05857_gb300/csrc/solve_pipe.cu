// solve_pipe.cu -- one epoch of BCPFW (pairwise steps, Alg. A.3, exact line
// search eq. 10) on a single instance with the LMO of the next block taken
// while the current block is being updated.
//
// A pairwise step of row i changes the plan, and so the residual r, in two
// columns only: the LMO vertex j* and the away vertex v. So the argmin of
// row i' = the row of the next update can be split exactly:
//   min over j not in {j*, v} of C_i'j + q_j   (q before the update: those
//                                               columns are unchanged by it)
//   and the two values at j*, v with the updated q.
// The compute warps take the first part for row p+1 while the control warp
// applies update p; the control warp then evaluates the two fresh values and
// merges them with the compute warps' partial minimum under the same order
// (value, then column), so the result is exactly the argmin over all
// columns at the updated residual, as in the non-pipelined kernel.
//
// Per phase p (one full barrier each):
//   compute warps: argmin of row p+1 over columns not in {j*_p, v_p} ->
//                  partials -> named barrier (arrive) -> cost row of p+2;
//   control warp:  decide and apply update p (atoms, plan, residual) ->
//                  away statistics of row p+1 at the new residual ->
//                  named barrier (wait) -> merge -> j*_{p+1}, exclusion set
//                  {j*_{p+1}, v_{p+1}} for the next phase.
// Compute warps read the residual while the control warp writes it, but only
// in the excluded columns, whose values they ignore.
//
// Layout, atom records (up to 63 per row, double-float weights), the
// compensated residual pair in shared memory, the record / cost-row ring
// (cp.async, D = RING - 2 rows ahead) and the overflow hand-off to the dense
// kernel are those of the active-set kernel (solve_sparse.cu).
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
__global__ void __launch_bounds__(NTC + kWarp, 1) k_epoch_pipe(EpochArgs<float> A) {
    constexpr int NWC = NTC / kWarp;  // compute warps; warp NWC is the control warp
    constexpr int NT = NTC + kWarp;
    constexpr int CPT = 4 * G;
    constexpr int WID = NTC * CPT;
    constexpr int D = RING - 2;
    static_assert(D >= 1, "ring too small");
    extern __shared__ __align__(16) unsigned char smem[];
    float *qh = reinterpret_cast<float *>(smem);
    float *ql = qh + WID;
    float4 *ys = reinterpret_cast<float4 *>(ql + WID);
    float *cring = reinterpret_cast<float *>(ys + (PTS ? WID : 0));
    int4 *aring = reinterpret_cast<int4 *>(cring + (PTS ? 0 : RING * WID));
    SpRed *red = reinterpret_cast<SpRed *>(aring + RING * kAtomRecord);
    int *sflag = reinterpret_cast<int *>(red + NWC);  // [0] stop, [2..3] exclusion set

    const int m = A.in.m, n = A.in.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool ctrl = warp == NWC;
    const unsigned FULL = 0xffffffffu;
    const float rho = (float)A.rho;
    const int order = A.order;
    const bool vec = A.vec;
    int4 *grec = A.atoms;
    const float INF = std::numeric_limits<float>::infinity();

    // ---- one-time set-up (as in the active-set kernel) --------------------
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
        sflag[0] = 0;
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
    auto fetch_async = [&](int i, int s) {
        if (ctrl) {
            cp16(aring + (size_t)s * kAtomRecord + lane, grec + (size_t)i * kAtomRecord + lane);
            cp16(aring + (size_t)s * kAtomRecord + 32 + lane, grec + (size_t)i * kAtomRecord + 32 + lane);
        } else if (!PTS) {
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
    // control warp: gradient of row (x, cost slot s) at column j, current residual
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
    // rq[t] = row of update p+1+t (t <= D); aq[t]: it travels by cp.async.
    // Row p+1+D is issued at the start of phase p; a row that repeats one of
    // the rows updated between its fetch and its use is loaded synchronously.
    int rq[D + 1];
    bool aq[D + 1];
    int row_cur = row_of(0);  // row of update p
    int row_prev = -1;        // row of update p-1 (its record writes precede this phase)
    // prologue: rows 0 .. D travel (row 0 in slot 0, ...)
    {
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
        // row 0 itself: its record and costs
        const bool ok0 = prefetchable && pre[0] >= 0;
        if (ctrl) {
            if (ok0) wait_groups<D>();
            else fetch_sync_record(pre[0], 0);
        } else if (!PTS) {
            if (ok0) wait_groups<D>();
            else fetch_sync_costs(pre[0], 0);
        }
    }
    // control state of the pending update (row_cur)
    float xc0 = 0.f, xc1 = 0.f, xc2 = 0.f, ac = 0.f;
    load_x(row_cur, xc0, xc1, xc2, ac);
    LaneAtoms at;
    AtomStats st;
    DF t_vdf{0.f, 0.f};
    float gmx = 0.f, inv = 0.f, gmin_cur = 0.f;
    int js_cur = 0;
    float xn0 = 0.f, xn1 = 0.f, xn2 = 0.f, an = 0.f;  // row of update p+1
    load_x(rq[0], xn0, xn1, xn2, an);

    // ---- prologue phase: LMO and away vertex of row 0 ---------------------
    __syncthreads();  // synchronous loads of row 0 visible
    if (!ctrl) {
        load_costs(0, xc0, xc1, xc2);
        partial_argmin(-1, -1);
        named_arrive(1, NT);
        if (m > 1) {
            if (!PTS) {
                if (aq[0]) wait_groups<D - 1>();
                else fetch_sync_costs(rq[0], 1 % RING);
            }
            load_costs(1 % RING, xn0, xn1, xn2);
        }
    } else {
        at = load_atoms(aring, lane);
        auto grad = [&](int j) -> float { return grad_at(j, 0, xc0, xc1, xc2); };
        st = atom_stats(at, grad, ac, false, &t_vdf);
        if (ac > 0.f) {
            gmx = st.t_v * (1.f / ac);  // same rounding as the two-phase kernel
            inv = 1.f / (2.f * rho * ac);
        }
        named_sync(1, NT);
        const SpRed e = lane < NWC ? red[lane] : SpRed{0xFFFFFFFFu, 0x7FFFFFFF};
        const uint32_t wk = __reduce_min_sync(FULL, e.kmin);
        js_cur = __reduce_min_sync(FULL, e.kmin == wk ? e.jmin : 0x7FFFFFFF);
        gmin_cur = key2f(wk);
        if (lane == 0) {
            if (!isfinite(gmin_cur)) {
                atomicCAS(A.status, 0, (int)kDevNonFinite);
                sflag[0] = 1;
            }
            sflag[2] = js_cur;
            sflag[3] = (st.v >= 0 && st.v < n) ? st.v : -1;
        }
    }
    __syncthreads();

    for (int p = 0; p < m && !sflag[0]; ++p) {
        const long long k = A.k0 + p;
        const bool more = p + 1 < m;
        const int row_p = row_cur;
        // issue row p+1+D (not if its record changes before it is used)
        {
            const int rnew = row_of(p + 1 + D);
            bool ok = prefetchable && rnew >= 0 && rnew != row_cur && rnew != row_prev;
#pragma unroll
            for (int u = 0; u < D; ++u) ok = ok && rnew != rq[u];
            if (ok) fetch_async(rnew, (p + 1 + D) % RING);
            commit();
            rq[D] = rnew;
            aq[D] = ok;
        }
        const int e1 = sflag[2], e2 = sflag[3];  // columns update p changes
        if (!ctrl) {
            if (more) {
                partial_argmin(e1, e2);
                named_arrive(1, NT);
                if (p + 2 < m) {
                    float xm0 = 0.f, xm1 = 0.f, xm2 = 0.f, am = 0.f;
                    load_x(rq[1], xm0, xm1, xm2, am);
                    if (!PTS) {
                        if (aq[1]) wait_groups<D - 1>();
                        else fetch_sync_costs(rq[1], (p + 2) % RING);
                    }
                    load_costs((p + 2) % RING, xm0, xm1, xm2);
                }
            }
        } else {
            // ---- update p -------------------------------------------------
            const int i = row_cur;
            bool present = false;
            int jpos = -1;
            atom_weight(at, js_cur, &present, &jpos);
            const Step<float> S = decide_pairwise(st, gmin_cur, js_cur, ac, rho, gmx, inv, n);
            bool ok = apply_pairwise(S, at, jpos, st.vpos, t_vdf, rho, A.T + (size_t)i * n, qh, ql,
                                     grec + (size_t)i * kAtomRecord, lane);
            if (lane == 0 && A.trace && k < A.trace_cap) {
                A.trace[4 * k] = i;
                A.trace[4 * k + 1] = js_cur;
                A.trace[4 * k + 2] = (st.v >= 0 && st.v < n) ? st.v : -1;
                A.trace[4 * k + 3] = __float_as_int(S.gamma);
            }
            if (!ok && lane == 0) {
                sflag[0] = 2;  // j* would be a 64th atom: the dense kernel takes over at p
                if (A.resume) *A.resume = p;
            }
            if (more) {
                // ---- row p+1: record, away vertex at the new residual ------
                const int i1 = rq[0];
                const int s1 = (p + 1) % RING;
                if (aq[0]) {
                    wait_groups<D>();
                } else {
                    __syncwarp();  // this warp's record writes of update p
                    fetch_sync_record(i1, s1);
                }
                __syncwarp();
                at = load_atoms(aring + (size_t)s1 * kAtomRecord, lane);
                auto grad = [&](int j) -> float { return grad_at(j, s1, xn0, xn1, xn2); };
                st = atom_stats(at, grad, an, false, &t_vdf);
                gmx = inv = 0.f;
                if (an > 0.f) {
                    gmx = st.t_v * (1.f / an);
                    inv = 1.f / (2.f * rho * an);
                }
                // ---- merge the compute warps' partial argmin ---------------
                named_sync(1, NT);
                const SpRed e = lane < NWC ? red[lane] : SpRed{0xFFFFFFFFu, 0x7FFFFFFF};
                uint32_t wk = __reduce_min_sync(FULL, e.kmin);
                int wj = __reduce_min_sync(FULL, e.kmin == wk ? e.jmin : 0x7FFFFFFF);
                // the columns update p changed, at the updated residual
                uint32_t kx = 0xFFFFFFFFu;
                int jx = 0x7FFFFFFF;
                const int ec = lane == 0 ? e1 : (lane == 1 ? e2 : -1);
                if (ec >= 0) {
                    kx = f2key(grad_at(ec, s1, xn0, xn1, xn2));
                    jx = ec;
                }
                if (kx < wk || (kx == wk && jx < wj)) { wk = kx; wj = jx; }
                const uint32_t fk = __reduce_min_sync(FULL, wk);
                js_cur = __reduce_min_sync(FULL, wk == fk ? wj : 0x7FFFFFFF);
                gmin_cur = key2f(fk);
                if (lane == 0) {
                    if (!isfinite(gmin_cur)) {
                        atomicCAS(A.status, 0, (int)kDevNonFinite);
                        sflag[0] = 1;
                    }
                    sflag[2] = js_cur;
                    sflag[3] = (st.v >= 0 && st.v < n) ? st.v : -1;
                }
                xc0 = xn0; xc1 = xn1; xc2 = xn2; ac = an;
            }
        }
        __syncthreads();  // residual, records, partials, exclusion set and costs ready
        if (sflag[0]) break;
        // advance the row pipeline (all threads)
        row_prev = row_p;
        row_cur = rq[0];
#pragma unroll
        for (int t = 0; t < D; ++t) { rq[t] = rq[t + 1]; aq[t] = aq[t + 1]; }
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, ta = 0.f;
        load_x(rq[0], t0, t1, t2, ta);
        xn0 = t0; xn1 = t1; xn2 = t2; an = ta;
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
    kern<<<1, NT + kWarp, pipe_smem<NT, G, PTS>(RING), st>>>(A);
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
