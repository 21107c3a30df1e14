// atoms.cuh -- the control warp of the active-set kernels: one row's atom
// record (active set S_i with double-float weights, up to 63 atoms, two per
// lane), the away vertex, the step decision and the update of atoms,
// residual and dense plan. Shared by the single-instance and batched kernels.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "step.cuh"

namespace srot {

// Record layout: entry 0 = {count, 0, 0, 0}; entry 1+k = atom k =
// {column, weight hi bits, weight lo bits, 0}. Lane l holds atoms l (slot 0)
// and 32+l (slot 1).
constexpr int kAtomsMax = kAtomRecord - 1;

struct LaneAtoms {
    int cnt;
    int j[2];
    DF t[2];
    float g[2];
};

// Load lane-local atoms from a record in shared or global memory.
__device__ inline LaneAtoms load_atoms(const int4 *rec, int lane) {
    LaneAtoms A;
    A.cnt = rec[0].x;
    const int4 e0 = rec[1 + lane];
    const int4 e1 = rec[1 + (lane + 32 < kAtomsMax ? lane + 32 : 0)];
    const bool h0 = lane < A.cnt, h1 = lane + 32 < A.cnt;
    A.j[0] = h0 ? e0.x : -1;
    A.t[0] = h0 ? DF{__int_as_float(e0.y), __int_as_float(e0.z)} : DF{0.f, 0.f};
    A.j[1] = h1 ? e1.x : -1;
    A.t[1] = h1 ? DF{__int_as_float(e1.y), __int_as_float(e1.z)} : DF{0.f, 0.f};
    A.g[0] = A.g[1] = 0.f;
    return A;
}

// A row's record as raw entries (count, this lane's two atoms): loads that
// can be issued an update ahead and decoded with decode_atoms when used.
struct RawAtoms {
    int4 head, e0, e1;
};
__device__ inline RawAtoms fetch_atoms(const int4 *rec, int lane) {
    RawAtoms R;
    R.head = rec[0];
    R.e0 = rec[1 + lane];
    R.e1 = rec[1 + (lane + 32 < kAtomsMax ? lane + 32 : 0)];
    return R;
}
__device__ inline LaneAtoms decode_atoms(const RawAtoms &R, int lane) {
    LaneAtoms A;
    A.cnt = R.head.x;
    const bool h0 = lane < A.cnt, h1 = lane + 32 < A.cnt;
    A.j[0] = h0 ? R.e0.x : -1;
    A.t[0] = h0 ? DF{__int_as_float(R.e0.y), __int_as_float(R.e0.z)} : DF{0.f, 0.f};
    A.j[1] = h1 ? R.e1.x : -1;
    A.t[1] = h1 ? DF{__int_as_float(R.e1.y), __int_as_float(R.e1.z)} : DF{0.f, 0.f};
    A.g[0] = A.g[1] = 0.f;
    return A;
}

// Gradient statistics over the atoms (see AtomStats). grad(j) evaluates the
// row gradient of column j; ai is the row weight.
template <typename GradF>
__device__ inline AtomStats atom_stats(LaneAtoms &A, GradF grad, float ai, bool want_sums, DF *t_v_df) {
    const unsigned FULL = 0xffffffffu;
    const bool two = A.cnt > 32;  // warp-uniform: slot 1 holds atoms
    uint32_t kx = 0u;
    int jx = 0x7FFFFFFF;
    if (A.j[0] >= 0) {
        A.g[0] = grad(A.j[0]);
        kx = f2key(A.g[0]);
        jx = A.j[0];
    }
    if (two && A.j[1] >= 0) {
        A.g[1] = grad(A.j[1]);
        const uint32_t kk = f2key(A.g[1]);
        if (kk > kx || (kk == kx && A.j[1] < jx)) { kx = kk; jx = A.j[1]; }
    }
    AtomStats S;
    const uint32_t wkx = __reduce_max_sync(FULL, kx);
    S.v = __reduce_min_sync(FULL, kx == wkx ? jx : 0x7FFFFFFF);
    S.gmax = key2f(wkx);
    S.nnz = A.cnt;
    DF tv{0.f, 0.f};
    int vl = -1;
    {
        const unsigned mk = __ballot_sync(FULL, A.j[0] >= 0 && A.j[0] == S.v);
        if (mk) vl = __ffs(mk) - 1;
    }
    if (two) {
        const unsigned mk = __ballot_sync(FULL, A.j[1] >= 0 && A.j[1] == S.v);
        if (mk) vl = 32 + __ffs(mk) - 1;
    }
    {
        const int src = vl >= 0 ? (vl & 31) : 0, sl = vl >> 5;  // vl is warp-uniform
        const float h = __shfl_sync(FULL, sl ? A.t[1].hi : A.t[0].hi, src);
        const float l = __shfl_sync(FULL, sl ? A.t[1].lo : A.t[0].lo, src);
        if (vl >= 0) tv = DF{h, l};
    }
    *t_v_df = tv;
    S.t_v = tv.hi;
    S.vpos = vl;
    S.g_aw = S.s2 = S.dda = 0.f;
    if (want_sums) {
        float aw = 0.f, s2 = 0.f, dd = 0.f;
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (A.j[s] >= 0 && (s == 0 || two)) {
                const float t = A.t[s].hi;
                aw += t * (S.gmax - A.g[s]);
                s2 += t * t;
                const float dv = (A.j[s] == S.v) ? t - ai : t;
                dd += dv * dv;
            }
        S.g_aw = warp_sum(aw);
        S.s2 = warp_sum(s2);
        S.dda = warp_sum(dd);
    }
    return S;
}

// Weight of column js among the atoms (0 if absent) and whether it is one;
// *pos (optional) receives its position in the record (-1 if absent).
__device__ inline float atom_weight(const LaneAtoms &A, int js, bool *present, int *pos = nullptr) {
    const unsigned FULL = 0xffffffffu;
    int where = -1;
    {
        const unsigned mk = __ballot_sync(FULL, A.j[0] >= 0 && A.j[0] == js);
        if (mk) where = __ffs(mk) - 1;
    }
    if (A.cnt > 32) {
        const unsigned mk = __ballot_sync(FULL, A.j[1] >= 0 && A.j[1] == js);
        if (mk) where = 32 + __ffs(mk) - 1;
    }
    const int src = where >= 0 ? (where & 31) : 0;
    const float h = __shfl_sync(FULL, (where >> 5) > 0 ? A.t[1].hi : A.t[0].hi, src);
    *present = where >= 0;
    if (pos) *pos = where;
    return where < 0 ? 0.f : h;
}

// Pairwise step (Alg. A.3) on the atom record: only the atoms j* and v
// change, so only the lanes holding them work. The moved mass is added to j*
// (appended at the end of the record when it enters) and taken from v with
// double-float arithmetic as in apply_atoms; an atom whose weight reaches 0
// is removed by moving the last atom into its place (the record's order
// carries no meaning: every reduction over it is by column). Plan entries
// and the residual pair change exactly as in apply_atoms.
//
// In three parts, for kernels that hand the new residual to another warp
// before they store it: pairwise_plan (new weights; 0: nothing changes, 1: a
// step, -1: j* would be atom 64 and nothing may change), pairwise_residual
// (lane 0: column j*, lane 1: column v; the new compensated residual pair
// from the current one), pairwise_store (plan entries and record).
struct PairStep {
    DF tj_old, tj_new, tv_new;
    int jpos, vpos;  // record positions of j* (-1 if absent) and v
    bool grows, append;
};
__device__ inline int pairwise_plan(const Step<float> &S, const LaneAtoms &A, int jpos, int vpos, DF t_v,
                                    PairStep *P) {
    const unsigned FULL = 0xffffffffu;
    if (S.kind != 2 || S.v == S.js || vpos < 0) return 0;
    P->jpos = jpos;
    P->vpos = vpos;
    P->grows = S.add_js > 0.f;
    P->append = P->grows && jpos < 0;
    if (P->append && A.cnt >= kAtomsMax) return -1;
    const DF mv = S.drop ? t_v : DF{S.add_js, 0.f};
    // old weight of j*, from the lane holding it
    const int jsrc = jpos >= 0 ? (jpos & 31) : 0;
    const float jh = __shfl_sync(FULL, (jpos >> 5) > 0 ? A.t[1].hi : A.t[0].hi, jsrc);
    const float jl = __shfl_sync(FULL, (jpos >> 5) > 0 ? A.t[1].lo : A.t[0].lo, jsrc);
    P->tj_old = jpos >= 0 ? DF{jh, jl} : DF{0.f, 0.f};
    P->tj_new = P->grows ? df_add(P->tj_old, mv) : P->tj_old;
    P->tv_new = S.drop ? DF{0.f, 0.f} : df_add(t_v, DF{-mv.hi, -mv.lo});
    return 1;
}
// Lanes 0 and 1 (others: *chg = false): the lane's column, whether its plan
// entry changes, and the residual pair after the step from the current pair
// (qc, lc) of that column.
__device__ inline void pairwise_residual(const PairStep &P, const Step<float> &S, DF t_v, float rho, int lane,
                                         float qc, float lc, int *col, bool *chg, float *qn, float *ln) {
    *col = lane == 0 ? S.js : S.v;
    const DF told = lane == 0 ? P.tj_old : t_v;
    const DF tn = lane == 0 ? P.tj_new : P.tv_new;
    *chg = lane < 2 && (tn.hi != told.hi || tn.lo != told.lo);
    *qn = qc;
    *ln = lc;
    if (*chg) {
        const float dlt = __fadd_rn(__fsub_rn(tn.hi, told.hi), __fsub_rn(tn.lo, told.lo));
        const float d = rho * dlt;
        const float y = __fsub_rn(d, lc);
        const float tt = __fadd_rn(qc, y);
        *ln = __fsub_rn(__fsub_rn(tt, qc), y);
        *qn = tt;
    }
}
__device__ inline void pairwise_store(const PairStep &P, const Step<float> &S, const LaneAtoms &A, DF t_v,
                                      float *trow, int4 *grec, int lane) {
    // plan entries: lane 0 takes j*, lane 1 takes v
    if (lane < 2) {
        const DF told = lane == 0 ? P.tj_old : t_v;
        const DF tn = lane == 0 ? P.tj_new : P.tv_new;
        if (tn.hi != told.hi || tn.lo != told.lo) trow[lane == 0 ? S.js : S.v] = tn.hi;
    }
    // record: positions of j* and v after the step
    int cnt = A.cnt;
    const int jp = P.append ? cnt : P.jpos;
    if (P.append) ++cnt;
    const bool vgone = !(P.tv_new.hi > 0.f);
    int4 *rec = grec + 1;
    if (lane == 0 && jp >= 0 && (P.grows || P.append))
        rec[jp] = make_int4(S.js, __float_as_int(P.tj_new.hi), __float_as_int(P.tj_new.lo), 0);
    if (!vgone) {
        if (lane == 1) rec[P.vpos] = make_int4(S.v, __float_as_int(P.tv_new.hi), __float_as_int(P.tv_new.lo), 0);
    } else {
        const int last = cnt - 1;
        if (last != P.vpos) {
            // move the last atom into v's place: j* (lane 0) when j* was just
            // appended, else the lane that holds the last atom writes it
            if (last == jp) {
                if (lane == 0)
                    rec[P.vpos] = make_int4(S.js, __float_as_int(P.tj_new.hi), __float_as_int(P.tj_new.lo), 0);
            } else if (lane == (last & 31)) {
                const int sl = last >> 5;
                rec[P.vpos] = make_int4(sl ? A.j[1] : A.j[0], __float_as_int(sl ? A.t[1].hi : A.t[0].hi),
                                        __float_as_int(sl ? A.t[1].lo : A.t[0].lo), 0);
            }
        }
        cnt = last;
    }
    if (lane == 0 && cnt != A.cnt) grec[0] = make_int4(cnt, 0, 0, 0);
}

// The whole step: jpos, vpos are the record positions of j* (-1 if absent)
// and v. Returns false (and changes nothing) if j* would be atom 64. mid()
// runs (on every lane, in every case that returns true) after the residual
// pair has changed and before the plan entries and the record are stored.
template <typename Mid>
__device__ inline bool apply_pairwise(const Step<float> &S, const LaneAtoms &A, int jpos, int vpos, DF t_v,
                                      float rho, float *trow, float *qh, float *ql, int4 *grec, int lane,
                                      Mid &&mid) {
    PairStep P;
    const int r = pairwise_plan(S, A, jpos, vpos, t_v, &P);
    if (r < 0) return false;
    if (r == 0) {
        mid();
        return true;
    }
    int col;
    bool chg;
    float qn, ln;
    const float qc = lane < 2 ? qh[lane == 0 ? S.js : S.v] : 0.f;
    const float lc = lane < 2 ? ql[lane == 0 ? S.js : S.v] : 0.f;
    pairwise_residual(P, S, t_v, rho, lane, qc, lc, &col, &chg, &qn, &ln);
    if (chg) {
        ql[col] = ln;
        qh[col] = qn;
    }
    mid();
    pairwise_store(P, S, A, t_v, trow, grec, lane);
    return true;
}

__device__ inline bool apply_pairwise(const Step<float> &S, const LaneAtoms &A, int jpos, int vpos, DF t_v,
                                      float rho, float *trow, float *qh, float *ql, int4 *grec, int lane) {
    return apply_pairwise(S, A, jpos, vpos, t_v, rho, trow, qh, ql, grec, lane, [] {});
}

// Apply step S of row i: atoms (with j* appended when it enters), dense
// plan entries, residual pair (qh, ql); writes the compacted record back to
// grec. Returns false (and changes nothing) if j* would be atom 64.
__device__ inline bool apply_atoms(const Step<float> &S, LaneAtoms &A, bool js_present, DF t_v, float ai,
                                   float rho, float *trow, float *qh, float *ql, int4 *grec, int lane) {
    const unsigned FULL = 0xffffffffu;
    if (S.kind < 0) return true;
    const bool grows = (S.kind == 0 || S.kind == 2) && S.add_js > 0.f;
    const bool append = grows && !js_present;
    if (append && A.cnt >= kAtomsMax) return false;
    const DF mv = (S.kind == 2 && S.drop) ? t_v : DF{S.add_js, 0.f};
    const bool two = A.cnt + (append ? 1 : 0) > 32;  // warp-uniform
    bool keep[2] = {false, false};
    DF tn[2];
    int jl[2] = {-1, -1};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (s == 1 && !two) break;
        const int k = lane + 32 * s;
        jl[s] = A.j[s];
        DF told = A.t[s];
        if (append && k == A.cnt) {
            jl[s] = S.js;
            told = DF{0.f, 0.f};
        }
        tn[s] = told;
        if (jl[s] >= 0) {
            tn[s] = apply_atom(S, jl[s], told, mv, ai);
            if (tn[s].hi != told.hi || tn[s].lo != told.lo) {
                trow[jl[s]] = tn[s].hi;
                const float dlt = __fadd_rn(__fsub_rn(tn[s].hi, told.hi), __fsub_rn(tn[s].lo, told.lo));
                const float d = rho * dlt;
                const float y = __fsub_rn(d, ql[jl[s]]);
                const float tt = __fadd_rn(qh[jl[s]], y);
                ql[jl[s]] = __fsub_rn(__fsub_rn(tt, qh[jl[s]]), y);
                qh[jl[s]] = tt;
            }
        }
        keep[s] = jl[s] >= 0 && tn[s].hi > 0.f;
    }
    const unsigned k0 = __ballot_sync(FULL, keep[0]);
    const unsigned k1 = two ? __ballot_sync(FULL, keep[1]) : 0u;
    const unsigned lt = (1u << lane) - 1u;
    if (keep[0]) grec[1 + __popc(k0 & lt)] = make_int4(jl[0], __float_as_int(tn[0].hi), __float_as_int(tn[0].lo), 0);
    if (keep[1]) grec[1 + __popc(k0) + __popc(k1 & lt)] = make_int4(jl[1], __float_as_int(tn[1].hi), __float_as_int(tn[1].lo), 0);
    if (lane == 0) grec[0] = make_int4(__popc(k0) + __popc(k1), 0, 0, 0);
    return true;
}

// Pairwise step (Alg. A.3) from the away statistics: gmx = t_v / a_i and
// inv = 1 / (2 rho a_i) computed before the LMO vertex is known.
__device__ inline Step<float> decide_pairwise(const AtomStats &st, float gmin, int js, float ai, float rho,
                                              float gmx, float inv, int n) {
    Step<float> S{-1, 0.f, js, st.v, 1.f, 0.f, 0.f, false};
    if (!(ai > 0.f) || st.v < 0 || st.v >= n) return S;
    S.kind = 2;
    if (st.v == js) return S;
    const float num = st.gmax - gmin;
    float gam = 0.f;
    if (num > 0.f) gam = rho > 0.f ? fminf(num * inv, gmx) : gmx;
    S.gamma = gam;
    S.drop = gam >= gmx;
    const float moved = S.drop ? st.t_v : gam * ai;
    S.add_js = moved;
    S.sub_v = moved;
    return S;
}

}  // namespace srot
