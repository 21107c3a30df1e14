// solve_batched.cu -- many independent instances of uneven size in one
// persistent launch (FP32, points with d = 3).
//
// Each CTA pulls instances from a device work queue (largest first) and
// solves each one to its stopping rule on its own: initial plan (Thm 1),
// epochs of block updates (Alg. 1 / A.2 / A.3 with the chosen order), and
// every `gap_every` epochs the certificate of Thm 2 taken inside the CTA
// (exact column sums of the plan, one LMO per row, compensated sums), which
// also reloads the running residual. No instance waits for another and the
// host is not involved until every instance is done.
//
// Per block update the CTA uses the active-set scheme of the single-instance
// kernel: compute warps own columns (target points in registers, residual as
// a compensated pair in shared memory) and run the LMO argmin; a control warp
// owns the row's atom record (up to 63 active atoms, two per lane), finds the
// away vertex, decides the step and applies it to the atoms, the residual and
// the dense plan. A row that would need a 64th atom stops its instance with
// kInstNeedsDense; the host then re-solves that instance on the dense path.
#include <algorithm>
#include <limits>
#include <vector>

#include "atoms.cuh"
#include "batched.h"
#include "common.cuh"
#include "cpasync.cuh"
#include "internal.h"
#include "step.cuh"

namespace srot {

namespace {

constexpr int kSmemMax = 227 * 1024;
constexpr int kPermMax = 2048;  // PERMUTE order: rows sorted in shared memory
constexpr int kRowMax = 2048;   // rows whose a_i and reciprocals are staged in shared memory

struct BRed {
    uint32_t kmin;
    int jmin;
};

__device__ inline float cost3f(float x0, float x1, float x2, float4 y) {
    const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
    return fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0)));
}

__device__ inline bool kv_less_b(uint64_t ka, int ia, uint64_t kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

}  // namespace

// Shared-memory bytes of one CTA for a tile of NTC compute threads x G quads.
template <int NTC, int G>
size_t batched_smem() {
    constexpr int WID = NTC * 4 * G;
    size_t b = 2 * (size_t)WID * 4;                  // qh, ql
    b += (size_t)WID * 16;                           // y table
    b += (size_t)kPermMax * (8 + 4);                 // permutation keys and rows
    b += 2 * ((NTC / kWarp) + 1) * sizeof(BRed);     // reduction slots
    b += 64 * sizeof(double) + 64;                   // certificate partials, flags
    b += (size_t)kRowMax * 16;                       // per-row a, 1/a, 1/(2 rho a)
    b += 4 * (size_t)kAtomRecord * 16;               // four-slot atom-record ring
    return b;
}

template <int NTC, int G>
__global__ void __launch_bounds__(NTC + kWarp, 1) k_batched(BatchArgs B) {
    constexpr int NWC = NTC / kWarp;
    constexpr int NW = NWC + 1;
    constexpr int NT = NTC + kWarp;
    constexpr int CPT = 4 * G;
    constexpr int WID = NTC * CPT;
    extern __shared__ __align__(16) unsigned char smem[];
    float *qh = reinterpret_cast<float *>(smem);
    float *ql = qh + WID;
    float4 *ys = reinterpret_cast<float4 *>(ql + WID);
    uint64_t *pkey = reinterpret_cast<uint64_t *>(ys + WID);
    int *prow = reinterpret_cast<int *>(pkey + kPermMax);
    BRed(*red)[NW] = reinterpret_cast<BRed(*)[NW]>(prow + kPermMax);
    double *cacc = reinterpret_cast<double *>(red + 2);  // certificate partials [NW][3]
    int *sflag = reinterpret_cast<int *>(cacc + 64);
    // per row {a_i, 1 / a_i, 1 / (2 rho a_i)}: the control warp reads them
    // from shared memory instead of loading and dividing on its chain
    float4 *arow = reinterpret_cast<float4 *>(sflag + 16);
    // atom records of the current and the next two rows (slot = update % 4),
    // streamed by compute warp 0
    int4 *aring = reinterpret_cast<int4 *>(arow + kRowMax);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool ctrl = warp == NWC;
    const unsigned FULL = 0xffffffffu;
    const float rho = (float)B.rho;
    const double rho64 = B.rho;

    for (;;) {
        __syncthreads();
        if (tid == 0) sflag[1] = atomicAdd(B.queue_head, 1);
        __syncthreads();
        const int qi = sflag[1];
        if (qi >= B.queue_len) break;
        const int inst = B.queue[qi];
        const BatchInst I = B.inst[inst];
        const int m = I.m, n = I.n;
        const float *X = B.X + I.off_X;
        const float *Y = B.Y + I.off_Y;
        const float *a = B.a + I.off_a;
        const float *b = B.b + I.off_b;
        float *T = B.T + I.off_T;
        int4 *grec = B.atoms + I.off_atoms;

        // ---- initial plan: T0 = (a_i e_0) (Thm 1), or the caller's plan -----
        // (warm start); atom records; residual
        if (tid == 0) sflag[0] = 0;
        if (!B.warm) {
            for (size_t e = tid; e < (size_t)m * n; e += NT) {
                const int i = (int)(e / n), j = (int)(e - (size_t)i * n);
                T[e] = j == 0 ? a[i] : 0.f;
            }
            for (int i = tid; i < m; i += NT) {
                const float ai = a[i];
                grec[(size_t)i * kAtomRecord] = make_int4(ai > 0.f ? 1 : 0, 0, 0, 0);
                grec[(size_t)i * kAtomRecord + 1] = make_int4(0, __float_as_int(ai), 0, 0);
            }
        }
        for (int i = tid; i < m && i < kRowMax; i += NT) {
            const float ai = a[i];
            arow[i] = make_float4(ai, ai > 0.f ? 1.f / ai : 0.f, ai > 0.f ? 1.f / (2.f * rho * ai) : 0.f, 0.f);
        }
        // s_0 = sum_i a_i in ascending order (one thread): the plan's total mass
        if (tid == 0) {
            double s0 = 0.0;
            for (int i = 0; i < m; ++i) s0 += (double)a[i];
            cacc[0] = s0;
        }
        __syncthreads();
        if (B.warm) {
            // the records of the caller's plan: each row's non-zero entries in
            // column order (one warp per row); a row with more than 63 stops
            // the instance for the dense path
            for (int i = warp; i < m; i += NW) {
                const float *trow = T + (size_t)i * n;
                int4 *rec = grec + (size_t)i * kAtomRecord;
                int cnt = 0;
                for (int j0 = 0; j0 < n; j0 += kWarp) {
                    const int j = j0 + lane;
                    const float t = j < n ? trow[j] : 0.f;
                    const unsigned mk = __ballot_sync(FULL, t > 0.f);
                    const int pos = cnt + __popc(mk & ((1u << lane) - 1u));
                    if (t > 0.f && pos < kAtomsMax) rec[1 + pos] = make_int4(j, __float_as_int(t), 0, 0);
                    cnt += __popc(mk);
                }
                if (lane == 0) {
                    rec[0] = make_int4(cnt <= kAtomsMax ? cnt : 0, 0, 0, 0);
                    if (cnt > kAtomsMax) sflag[0] = kInstNeedsDense;
                }
            }
            __syncthreads();
        }
        const int init_flag = sflag[0];
        // fixed-point exponent for the certificate's column sums (see there)
        int fx_exp;
        {
            int e2 = 0;
            frexp(cacc[0] > 1.0 ? cacc[0] : 1.0, &e2);  // total mass < 2^e2
            fx_exp = 61 - e2;
        }
        for (int j = tid; j < WID; j += NT) {
            if (j < n) {
                double sj = j == 0 ? cacc[0] : 0.0;
                if (B.warm) {  // the plan's column sum, rows in ascending order
                    sj = 0.0;
                    for (int i = 0; i < m; ++i) sj += (double)T[(size_t)i * n + j];
                }
                const double qq = rho64 * (sj - (double)b[j]);
                const float h = (float)qq;
                qh[j] = h;
                ql[j] = (float)((double)h - qq);
                ys[j] = make_float4(Y[(size_t)j * 3], Y[(size_t)j * 3 + 1], Y[(size_t)j * 3 + 2], 0.f);
            } else {
                qh[j] = 1e30f;
                ql[j] = 0.f;
                ys[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float2 ny0[2 * G], ny1[2 * G], ny2[2 * G];
        if (!ctrl) {
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = 4 * (tid + NTC * g) + 2 * h;
                    const bool a0 = j < n, a1 = j + 1 < n;
                    ny0[2 * g + h] = make_float2(a0 ? -Y[(size_t)j * 3] : 0.f, a1 ? -Y[(size_t)(j + 1) * 3] : 0.f);
                    ny1[2 * g + h] = make_float2(a0 ? -Y[(size_t)j * 3 + 1] : 0.f, a1 ? -Y[(size_t)(j + 1) * 3 + 1] : 0.f);
                    ny2[2 * g + h] = make_float2(a0 ? -Y[(size_t)j * 3 + 2] : 0.f, a1 ? -Y[(size_t)(j + 1) * 3 + 2] : 0.f);
                }
        }
        __syncthreads();

        double f = 0.0, gap = 0.0, feas_err = 0.0;
        long long ep = 0, updates = 0;
        long long next_cert = 0;  // epoch count at which the next certificate is due
        int status = kInstOk;
        int par = 0;
        if (init_flag) status = init_flag;
        for (ep = 0; !init_flag && ep < B.max_epochs; ++ep) {
            const long long k0 = ep * (long long)m;
            // ---- block order of this epoch --------------------------------
            if (B.order == SR_OT_PERMUTE) {
                int L = 1;
                while (L < m) L <<= 1;
                for (int t = tid; t < L; t += NT) {
                    if (t < m) {
                        pkey[t] = sm64_draw(B.seed, 1, (uint64_t)ep * (uint64_t)m + (uint64_t)t);
                        prow[t] = t;
                    } else {
                        pkey[t] = ~0ULL;
                        prow[t] = 0x7FFFFFFF;
                    }
                }
                __syncthreads();
                for (int kk = 2; kk <= L; kk <<= 1)
                    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                        for (int t = tid; t < L; t += NT) {
                            const int l = t ^ jj;
                            if (l > t) {
                                const bool up = (t & kk) == 0;
                                const uint64_t kt = pkey[t], kl = pkey[l];
                                const int it = prow[t], il = prow[l];
                                const bool sw = up ? kv_less_b(kl, il, kt, it) : kv_less_b(kt, it, kl, il);
                                if (sw) { pkey[t] = kl; pkey[l] = kt; prow[t] = il; prow[l] = it; }
                            }
                        }
                        __syncthreads();
                    }
            }
            auto row_of = [&](int p) -> int {
                if (B.order == SR_OT_CYCLIC) return p;
                if (B.order == SR_OT_PERMUTE) return prow[p];
                return scale_u64(sm64_draw(B.seed, 2, (uint64_t)(k0 + p)), m);
            };

            // ---- m block updates ---------------------------------------------
            float cst[CPT];
            int i_next = row_of(0);
            // atom records: row of update p in ring slot p & 3; compute warp 0
            // streams the record of update p + 2 during update p, unless that
            // row is updated before its use (the rows of updates p, p + 1)
            int i_p1 = m > 1 ? row_of(1) : -1;
            bool pre_cur = true;                    // the current row's record is in its slot
            int i_prev = -1;                        // the row of update p - 1
            bool pre_next = i_p1 >= 0 && i_p1 != i_next;  // the next one's
            if (warp == 0) {
                cp16(aring + lane, grec + (size_t)i_next * kAtomRecord + lane);
                cp16(aring + 32 + lane, grec + (size_t)i_next * kAtomRecord + 32 + lane);
                commit();
                if (pre_next) {
                    cp16(aring + kAtomRecord + lane, grec + (size_t)i_p1 * kAtomRecord + lane);
                    cp16(aring + kAtomRecord + 32 + lane, grec + (size_t)i_p1 * kAtomRecord + 32 + lane);
                }
                commit();
                wait_groups<1>();  // row 0's record
            }
            float xn0 = 0.f, xn1 = 0.f, xn2 = 0.f;
            xn0 = X[(size_t)i_next * 3];
            xn1 = X[(size_t)i_next * 3 + 1];
            xn2 = X[(size_t)i_next * 3 + 2];
            // x of the row two updates ahead, loaded an update before its use
            int i_far = m > 1 ? row_of(1) : -1;
            float xf0 = 0.f, xf1 = 0.f, xf2 = 0.f;
            if (i_far >= 0) {
                xf0 = X[(size_t)i_far * 3];
                xf1 = X[(size_t)i_far * 3 + 1];
                xf2 = X[(size_t)i_far * 3 + 2];
            }
            if (!ctrl) {
                const float2 X0 = make_float2(xn0, xn0), X1 = make_float2(xn1, xn1), X2 = make_float2(xn2, xn2);
#pragma unroll
                for (int hh = 0; hh < 2 * G; ++hh) {
                    const float2 d0 = __fadd2_rn(X0, ny0[hh]), d1 = __fadd2_rn(X1, ny1[hh]), d2 = __fadd2_rn(X2, ny2[hh]);
                    float2 c = __fmul2_rn(d0, d0);
                    c = __ffma2_rn(d1, d1, c);
                    c = __ffma2_rn(d2, d2, c);
                    cst[2 * hh] = c.x;
                    cst[2 * hh + 1] = c.y;
                }
            }
            __syncthreads();  // row 0's record visible
            for (int p = 0; p < m; ++p) {
                const long long k = k0 + p;
                const int i = i_next;
                const float x0 = xn0, x1 = xn1, x2 = xn2;
                const int slot = p & 3;
                if (p + 1 < m) {
                    i_next = i_far;
                    xn0 = xf0;
                    xn1 = xf1;
                    xn2 = xf2;
                    i_far = p + 2 < m ? row_of(p + 2) : -1;
                    if (i_far >= 0) {
                        xf0 = X[(size_t)i_far * 3];
                        xf1 = X[(size_t)i_far * 3 + 1];
                        xf2 = X[(size_t)i_far * 3 + 2];
                    }
                }
                AtomStats st{};
                DF t_vdf{0.f, 0.f};
                float ai = 0.f, gmx = 0.f, inv = 0.f;
                LaneAtoms at_cur;
                // the record of update p + 2 travels unless that row is
                // rewritten just before the copy or before its use (updates
                // p - 1, p, p + 1)
                const bool pre_far = p + 2 < m && i_far != i && i_far != i_next && i_far != i_prev;
                if (warp == 0) {
                    if (pre_far) {
                        int4 *dst = aring + (size_t)((p + 2) & 3) * kAtomRecord;
                        cp16(dst + lane, grec + (size_t)i_far * kAtomRecord + lane);
                        cp16(dst + 32 + lane, grec + (size_t)i_far * kAtomRecord + 32 + lane);
                    }
                    commit();
                }
                if (!ctrl) {
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
                    const uint32_t km = f2key(qv[0]);
                    const uint32_t wk = __reduce_min_sync(FULL, km);
                    const int wj = __reduce_min_sync(FULL, km == wk ? qj[0] : 0x7FFFFFFF);
                    if (lane == 0) red[par][warp] = BRed{wk, wj};
                } else {
                    int4 *rec = aring + (size_t)slot * kAtomRecord;
                    if (!pre_cur) {
                        rec[lane] = grec[(size_t)i * kAtomRecord + lane];
                        rec[32 + lane] = grec[(size_t)i * kAtomRecord + 32 + lane];
                        __syncwarp();
                    }
                    at_cur = load_atoms(rec, lane);
                    float ra, ia;
                    if (m <= kRowMax) {
                        const float4 ar = arow[i];
                        ai = ar.x;
                        ra = ar.y;
                        ia = ar.z;
                    } else {
                        ai = a[i];
                        ra = ai > 0.f ? 1.f / ai : 0.f;
                        ia = ai > 0.f ? 1.f / (2.f * rho * ai) : 0.f;
                    }
                    auto grad = [&](int j) -> float { return cost3f(x0, x1, x2, ys[j]) + qh[j]; };
                    st = atom_stats(at_cur, grad, ai, B.variant != SR_OT_BCPFW, &t_vdf);
                    if (B.variant == SR_OT_BCPFW && ai > 0.f) {
                        gmx = st.t_v * ra;  // gamma_max = alpha_v = t_v / a_i
                        inv = ia;           // eq. 10 with d = a_i (e_j* - e_v)
                    }
                }
                __syncthreads();  // (A)
                if (ctrl) {
                    const BRed e = lane < NWC ? red[par][lane] : BRed{0xFFFFFFFFu, 0x7FFFFFFF};
                    const uint32_t wk = __reduce_min_sync(FULL, e.kmin);
                    const int js = __reduce_min_sync(FULL, e.kmin == wk ? e.jmin : 0x7FFFFFFF);
                    const float gmin_all = key2f(wk);
                    bool present = false;
                    int jpos = -1;
                    const float t_js = atom_weight(at_cur, js, &present, &jpos);
                    bool stop = false;
                    if (!isfinite(gmin_all)) {
                        if (lane == 0) sflag[0] = kInstNonFinite;
                        stop = true;
                    }
                    Step<float> S{-1, 0.f, js, st.v, 1.f, 0.f, 0.f, false};
                    if (!stop)
                        S = B.variant == SR_OT_BCPFW
                                ? decide_pairwise(st, gmin_all, js, ai, rho, gmx, inv, n)
                                : decide_atoms(st, gmin_all, js, t_js, ai, B.variant, B.step, rho, m, k);
                    const bool applied =
                        stop || (B.variant == SR_OT_BCPFW
                                     ? apply_pairwise(S, at_cur, jpos, st.vpos, t_vdf, rho, T + (size_t)i * n, qh,
                                                      ql, grec + (size_t)i * kAtomRecord, lane)
                                     : apply_atoms(S, at_cur, present, t_vdf, ai, rho, T + (size_t)i * n, qh, ql,
                                                   grec + (size_t)i * kAtomRecord, lane));
                    if (!applied) {
                        if (lane == 0) sflag[0] = kInstNeedsDense;
                    }

                } else if (p + 1 < m) {
                    const float2 X0 = make_float2(xn0, xn0), X1 = make_float2(xn1, xn1), X2 = make_float2(xn2, xn2);
#pragma unroll
                    for (int hh = 0; hh < 2 * G; ++hh) {
                        const float2 d0 = __fadd2_rn(X0, ny0[hh]), d1 = __fadd2_rn(X1, ny1[hh]), d2 = __fadd2_rn(X2, ny2[hh]);
                        float2 c = __fmul2_rn(d0, d0);
                        c = __ffma2_rn(d1, d1, c);
                        c = __ffma2_rn(d2, d2, c);
                        cst[2 * hh] = c.x;
                        cst[2 * hh + 1] = c.y;
                    }
                }
                if (warp == 0) wait_groups<1>();  // the next row's record (p + 2's may be in flight)
                par ^= 1;
                __syncthreads();  // (B)
                if (sflag[0]) break;
                ++updates;
                pre_cur = pre_next;
                pre_next = pre_far;
                i_prev = i;
            }
            if (warp == 0) wait_groups<0>();  // a record copy may still be in flight after an early stop
            if (sflag[0]) { status = sflag[0]; break; }

            // ---- certificate (Thm 2) ------------------------------------------
            // every gap_every epochs and at the end; while the last relative gap
            // was far above the tolerance the next one is taken later (each
            // costs two passes over the plan at one SM's share of bandwidth)
            const bool last = ep + 1 == B.max_epochs;
            if (!((ep + 1) % B.gap_every == 0 || last)) continue;
            if (!last && ep + 1 < next_cert) continue;
            // exact column sums s_j from the atom records (the plan's nonzeros,
            // with their double-float weights) as 64-bit fixed-point integers:
            // integer addition is exact, so the order in which threads add does
            // not change the result. Scale: 2^fx_exp with every column sum below
            // the total mass sum_i a_i < 2^(62 - fx_exp).
            {
                unsigned long long *csum = reinterpret_cast<unsigned long long *>(pkey);  // n <= kPermMax
                for (int j = tid; j < n; j += NT) csum[j] = 0ull;
                __syncthreads();
                // one row per thread: many records in flight at once
                for (int i = tid; i < m; i += NT) {
                    const int4 *g = grec + (size_t)i * kAtomRecord;
                    const int4 h0 = g[0], e0 = g[1];
                    const int c = h0.x;
                    for (int kk = 0; kk < c; ++kk) {
                        const int4 at = kk == 0 ? e0 : g[1 + kk];
                        const double t = (double)__int_as_float(at.y) + (double)__int_as_float(at.z);
                        if (t > 0.0)
                            atomicAdd(&csum[at.x], (unsigned long long)__double2ll_rn(ldexp(t, fx_exp)));
                    }
                }
                __syncthreads();
                for (int j = tid; j < n; j += NT) {
                    const double sj = ldexp((double)(long long)csum[j], -fx_exp);
                    const double qq = rho64 * (sj - (double)b[j]);
                    const float h = (float)qq;
                    qh[j] = h;  // refresh of the running residual
                    ql[j] = (float)((double)h - qq);
                }
            }
            __syncthreads();
            // per row: LMO vertex over all columns, <t_i, c_i>, <t_i, q>
            double lin = 0.0, tq = 0.0, amin = 0.0, feas = 0.0;
            if (m <= kRowMax) {
                // (a) the LMO: one warp per row over the columns (x of the
                // warp's next row loaded while this one is processed)
                int i = warp;
                float xi0 = 0.f, xi1 = 0.f, xi2 = 0.f;
                if (i < m) { xi0 = X[(size_t)i * 3]; xi1 = X[(size_t)i * 3 + 1]; xi2 = X[(size_t)i * 3 + 2]; }
                for (; i < m; i += NW) {
                    const int inx = i + NW;
                    float nx0 = 0.f, nx1 = 0.f, nx2 = 0.f;
                    if (inx < m) { nx0 = X[(size_t)inx * 3]; nx1 = X[(size_t)inx * 3 + 1]; nx2 = X[(size_t)inx * 3 + 2]; }
                    float gb = std::numeric_limits<float>::infinity();
                    int jb = 0x7FFFFFFF;
                    for (int j = lane; j < n; j += kWarp) {
                        const float gr = cost3f(xi0, xi1, xi2, ys[j]) + qh[j];
                        if (gr < gb || jb == 0x7FFFFFFF) { gb = gr; jb = j; }
                    }
                    const uint32_t kb = f2key(gb);
                    const uint32_t wk = __reduce_min_sync(FULL, kb);
                    const int jm = __reduce_min_sync(FULL, kb == wk ? jb : 0x7FFFFFFF);
                    if (lane == 0) arow[i].w = __int_as_float(jm);
                    xi0 = nx0; xi1 = nx1; xi2 = nx2;
                }
                __syncthreads();
                // (b) per row, one row per thread: a_i min_j grad_ij at the LMO
                // vertex, and the atom sums <t_i, c_i>, <t_i, q>, sum_j t_ij
                for (int r = tid; r < m; r += NT) {
                    const float y0 = X[(size_t)r * 3], y1 = X[(size_t)r * 3 + 1], y2 = X[(size_t)r * 3 + 2];
                    const int jm = __float_as_int(arow[r].w);
                    const int4 *g = grec + (size_t)r * kAtomRecord;
                    const int c = g[0].x;
                    double l1 = 0.0, l2 = 0.0, l3 = 0.0;
                    for (int kk = 0; kk < c; ++kk) {
                        const int4 at = g[1 + kk];
                        const double t = (double)__int_as_float(at.y) + (double)__int_as_float(at.z);
                        l1 += t * (double)cost3f(y0, y1, y2, ys[at.x]);
                        l2 += t * ((double)qh[at.x] - (double)ql[at.x]);
                        l3 += t;
                    }
                    const double gmin = (double)cost3f(y0, y1, y2, ys[jm]) + ((double)qh[jm] - (double)ql[jm]);
                    const double ai = (double)arow[r].x;
                    lin += l1;
                    tq += l2;
                    amin += ai * gmin;
                    feas = fmax(feas, fabs(l3 - ai) / (ai > 0.0 ? ai : 1e-300));
                }
                lin = warp_sum(lin);
                tq = warp_sum(tq);
                amin = warp_sum(amin);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) feas = fmax(feas, __shfl_xor_sync(FULL, feas, o));
            } else
            for (int i = warp; i < m; i += NW) {
                const float xi0 = X[(size_t)i * 3], xi1 = X[(size_t)i * 3 + 1], xi2 = X[(size_t)i * 3 + 2];
                float gb = std::numeric_limits<float>::infinity();
                int jb = 0x7FFFFFFF;
                for (int j = lane; j < n; j += kWarp) {
                    const float gr = cost3f(xi0, xi1, xi2, ys[j]) + qh[j];
                    if (gr < gb || jb == 0x7FFFFFFF) { gb = gr; jb = j; }
                }
                const uint32_t kb = f2key(gb);
                const uint32_t wk = __reduce_min_sync(FULL, kb);
                const int jm = __reduce_min_sync(FULL, kb == wk ? jb : 0x7FFFFFFF);
                // atoms of row i
                const int4 *g = grec + (size_t)i * kAtomRecord;
                const int c = g[0].x;
                double l1 = 0.0, l2 = 0.0, l3 = 0.0;
                for (int kk = lane; kk < c; kk += kWarp) {
                    const int4 at = g[1 + kk];
                    const double t = (double)__int_as_float(at.y) + (double)__int_as_float(at.z);
                    l1 += t * (double)cost3f(xi0, xi1, xi2, ys[at.x]);
                    l2 += t * ((double)qh[at.x] - (double)ql[at.x]);
                    l3 += t;
                }
                l1 = warp_sum(l1);
                l2 = warp_sum(l2);
                l3 = warp_sum(l3);
                if (lane == 0) {
                    const double gmin = (double)cost3f(xi0, xi1, xi2, ys[jm]) + ((double)qh[jm] - (double)ql[jm]);
                    const double ai = (double)a[i];
                    lin += l1;
                    tq += l2;
                    amin += ai * gmin;
                    feas = fmax(feas, fabs(l3 - ai) / (ai > 0.0 ? ai : 1e-300));
                }
            }
            if (lane == 0) {
                cacc[3 * warp] = lin;
                cacc[3 * warp + 1] = tq;
                cacc[3 * warp + 2] = amin;
                cacc[40 + warp] = feas;
            }
            double rr = 0.0;
            for (int j = tid; j < n; j += NT) {
                const double qq = (double)qh[j] - (double)ql[j];
                rr += qq * qq;
            }
            rr = warp_sum(rr);
            __syncthreads();
            if (lane == 0) cacc[3 * NW + warp] = rr;
            __syncthreads();
            if (tid == 0) {
                double L = 0.0, Q = 0.0, A2 = 0.0, R2 = 0.0, FE = 0.0;
                for (int w = 0; w < NW; ++w) {
                    L += cacc[3 * w];
                    Q += cacc[3 * w + 1];
                    A2 += cacc[3 * w + 2];
                    R2 += cacc[3 * NW + w];
                    FE = fmax(FE, cacc[40 + w]);
                }
                cacc[62] = FE;
                // q = rho r: ||r||^2 = R2 / rho^2, <t, grad> summed = L + Q
                const double pen = rho64 > 0.0 ? 0.5 * R2 / rho64 : 0.0;
                cacc[60] = L + pen;           // f
                cacc[61] = (L + Q) - A2;      // g
            }
            __syncthreads();
            f = cacc[60];
            gap = cacc[61];
            feas_err = cacc[62];
            if (B.tol > 0.0 && gap <= B.tol * f && feas_err <= kFeasTol) { ++ep; break; }
            if (B.tol > 0.0) {
                const double rel = f > 0.0 ? gap / f : 0.0;
                const long long skip = rel > 1000.0 * B.tol ? 8 : (rel > 100.0 * B.tol ? 4 : (rel > 10.0 * B.tol ? 2 : 1));
                next_cert = ep + 1 + skip * B.gap_every;
            }
        }
        if (status == kInstOk && B.tol > 0.0 && !(gap <= B.tol * f && feas_err <= kFeasTol))
            status = kInstNotConverged;
        if (tid == 0) {
            BatchResult &r = B.res[inst];
            r.f = f;
            r.g = gap;
            r.feas = feas_err;
            r.epochs = ep;
            r.updates = updates;
            r.status = status;
        }
    }
}

template <int NTC, int G>
static void launch_tile(const BatchArgs &B, int grid, cudaStream_t st) {
    auto kern = k_batched<NTC, G>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
        attr_set = true;
    }
    kern<<<grid, NTC + kWarp, batched_smem<NTC, G>(), st>>>(B);
}

const BatchTile kBatchTiles[] = {
    {64, 1}, {64, 2}, {128, 1}, {128, 2}, {64, 4}, {128, 4}, {256, 2},
};
const int kNumBatchTiles = sizeof(kBatchTiles) / sizeof(kBatchTiles[0]);

size_t batch_tile_smem(int t) {
    switch (t) {
        case 0: return batched_smem<64, 1>();
        case 1: return batched_smem<64, 2>();
        case 2: return batched_smem<128, 1>();
        case 3: return batched_smem<128, 2>();
        case 4: return batched_smem<64, 4>();
        case 5: return batched_smem<128, 4>();
        default: return batched_smem<256, 2>();
    }
}

void launch_batched_tile(int t, const BatchArgs &B, int grid, cudaStream_t st) {
    switch (t) {
        case 0: launch_tile<64, 1>(B, grid, st); break;
        case 1: launch_tile<64, 2>(B, grid, st); break;
        case 2: launch_tile<128, 1>(B, grid, st); break;
        case 3: launch_tile<128, 2>(B, grid, st); break;
        case 4: launch_tile<64, 4>(B, grid, st); break;
        case 5: launch_tile<128, 4>(B, grid, st); break;
        default: launch_tile<256, 2>(B, grid, st); break;
    }
}

int batch_tile_ctas_per_sm(int t) {
    const size_t sm = batch_tile_smem(t);
    const int threads = kBatchTiles[t].ntc + kWarp;
    int by_smem = (int)((228 * 1024) / (sm + 1024));
    int by_threads = 2048 / threads;
    return std::max(1, std::min(by_smem, by_threads));
}

}  // namespace srot
