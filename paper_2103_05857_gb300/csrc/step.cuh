// step.cuh -- the per-block decision shared by the dense and sparse epoch
// kernels: exact line search (eq. 8, eq. 10), the choice between FW, away and
// pairwise directions (Alg. 1, A.2, A.3), and the new value of one entry.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace srot {

// Squared-Euclidean cost of one (x_i, y_j) pair in d = 3. The FP32 form is
// the one every FP32 kernel (solver, certificate) evaluates, so all of them
// see the same cost matrix; the FP64 form uses the rounding order of the
// plain definition (no contraction).
__device__ inline float cost3(float x0, float x1, float x2, float y0, float y1, float y2) {
    float d0 = x0 - y0, d1 = x1 - y1, d2 = x2 - y2;
    return fmaf(d2, d2, fmaf(d1, d1, __fmul_rn(d0, d0)));
}
__device__ inline double cost3(double x0, double x1, double x2, double y0, double y1, double y2) {
    double d0 = dsub(x0, y0), d1 = dsub(x1, y1), d2 = dsub(x2, y2);
    return dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2));
}

// Block-wide result of one reduction (identical in every thread).
template <typename Real>
struct Red {
    Real gmin, s1, s2, gmax;
    int jmin, jmax, nnz;
    Real rs;  // FP32 away steps: sum_j t_ij as stored
};

// Exact line search on phi(gamma) = -num gamma + (rho/2) dd gamma^2, [0, gmax].
template <typename Real>
__device__ inline Real line_search(Real num, Real dd, Real rho, Real gmax) {
    if (!(num > Real(0))) return Real(0);
    Real den = rho * dd;
    if (!(den > Real(0))) return gmax;
    Real g = num / den;
    return g < gmax ? g : gmax;
}

// Decisions of one block update (identical in every thread).
template <typename Real>
struct Step {
    int kind;        // -1 none, 0 FW convex combination, 1 away, 2 pairwise
    Real gamma;
    int js, v;
    Real coef;       // FW: 1-gamma ; away: 1+gamma
    Real add_js;     // value added at j* (FW: gamma a_i ; pairwise: moved mass)
    Real sub_v;      // pairwise: moved mass ; away: gamma a_i
    bool drop;
};

// Unit in the last place of a nonnegative float (0 for 0; the smallest
// normal spacing below 2^-103).
__device__ inline float ulpf(float x) {
    const int e = __float_as_int(x) & 0x7F800000;
    if (e == 0) return 0.f;
    return e > (23 << 23) + (1 << 23) ? __int_as_float(e - (23 << 23)) : __int_as_float(1 << 23);
}

// Mass moved between two FP32 plan entries a and b (a gains, b loses),
// rounded to a multiple of the coarser spacing of the two so that both
// a + moved and b - moved are exact: otherwise a move below half an ulp of
// the larger entry is absorbed there but not at the other one, and the row
// mass drifts systematically over many small steps. Never exceeds b.
__device__ inline float conserving_move(float moved, float a, float b) {
    const float u = fmaxf(ulpf(a), ulpf(b));
    if (!(u > 0.f) || u < 0x1.0p-100f) return moved;
    const float inv = 1.f / u;  // a power of two: exact
    float q = rintf(moved * inv) * u;
    if (q > b) q = floorf(b * inv) * u;
    return q;
}

template <typename Real>
__device__ inline Step<Real> decide(const Red<Real> &R, Real ai, Real t_js, Real t_v, int variant,
                                    int step, Real rho, int m, long long k) {
    Step<Real> S;
    S.kind = -1; S.gamma = Real(0); S.js = R.jmin; S.v = R.jmax;
    S.coef = Real(1); S.add_js = Real(0); S.sub_v = Real(0); S.drop = false;
    if (!(ai > Real(0))) return S;
    const Real g_fw = R.s1 - ai * R.gmin;
    if (variant == SR_OT_BCFW) {
        Real gam;
        if (step == SR_OT_DEC) {
            if constexpr (std::is_same<Real, double>::value)
                gam = __ddiv_rn(2.0 * (double)m, (double)k + 2.0 * (double)m);
            else
                gam = (float)((2.0 * (double)m) / ((double)k + 2.0 * (double)m));
        } else {
            Real dd = (R.s2 - t_js * t_js) + (ai - t_js) * (ai - t_js);
            gam = line_search<Real>(g_fw, dd > Real(0) ? dd : Real(0), rho, Real(1));
        }
        S.kind = 0; S.gamma = gam;
        if constexpr (std::is_same<Real, double>::value) {
            S.coef = dsub(1.0, gam);
            S.add_js = dmul(gam, ai);
        } else {
            S.coef = 1.f - gam;
            S.add_js = gam * ai;
        }
        return S;
    }
    if (S.v < 0 || S.v == 0x7FFFFFFF) return S;
    if (variant == SR_OT_BCAFW) {
        const Real g_aw = ai * R.gmax - R.s1;
        // Mass of the other atoms: a_i - t_v in exact arithmetic. FP32 uses
        // the stored row minus t_v, so that the step conserves the row as
        // stored: with alpha_v near 1, gamma_max = alpha/(1-alpha) is huge
        // and a_i - t_v would multiply the row's rounding drift by it.
        Real s_oth;
        if constexpr (std::is_same<Real, float>::value) s_oth = R.rs - t_v;
        else s_oth = ai - t_v;
        // alpha_v >= 1 (all the mass on v): the away direction is zero
        if (R.nnz <= 1 || g_fw >= g_aw || !(s_oth > Real(0))) {
            Real dd = (R.s2 - t_js * t_js) + (ai - t_js) * (ai - t_js);
            Real gam = line_search<Real>(g_fw, dd > Real(0) ? dd : Real(0), rho, Real(1));
            S.kind = 0; S.gamma = gam; S.coef = Real(1) - gam; S.add_js = gam * ai;
        } else {
            Real gmax, dd;
            if constexpr (std::is_same<Real, float>::value) {
                gmax = t_v / s_oth;  // = alpha / (1 - alpha)
                dd = (R.s2 - t_v * t_v) + s_oth * s_oth;
            } else {
                const Real alpha = t_v / ai;
                gmax = alpha / (Real(1) - alpha);
                dd = (R.s2 - t_v * t_v) + (t_v - ai) * (t_v - ai);
            }
            Real gam = line_search<Real>(g_aw, dd > Real(0) ? dd : Real(0), rho, gmax);
            S.kind = 1; S.gamma = gam; S.coef = Real(1) + gam;
            // FP32: v loses gamma * s_oth directly; FP64: (1 + gamma) t_v - gamma a_i
            if constexpr (std::is_same<Real, float>::value) S.sub_v = gam * s_oth;
            else S.sub_v = gam * ai;
            S.drop = gam >= gmax;
        }
        return S;
    }
    // pairwise
    if (S.v == S.js) { S.kind = 2; return S; }
    Real g_pw = ai * (R.gmax - R.gmin);
    Real gmax = t_v / ai;
    Real gam = line_search<Real>(g_pw, Real(2) * ai * ai, rho, gmax);
    S.kind = 2; S.gamma = gam;
    S.drop = gam >= gmax;
    Real moved = S.drop ? t_v : gam * ai;
    if constexpr (std::is_same<Real, float>::value)
        if (!S.drop) moved = conserving_move(moved, t_js, t_v);
    S.add_js = moved; S.sub_v = moved;
    return S;
}

// New value of one owned entry under step S.
template <typename Real>
__device__ inline Real apply(const Step<Real> &S, int j, Real t) {
    if (S.kind == 0) {
        Real tn;
        if constexpr (std::is_same<Real, double>::value) {
            tn = dmul(S.coef, t);
            if (j == S.js) tn = dadd(tn, S.add_js);
        } else {
            tn = S.coef * t;
            if (j == S.js) tn = tn + S.add_js;
        }
        return tn;
    }
    if (S.kind == 1) {
        if (j == S.v) {
            if (S.drop) return Real(0);
            if constexpr (std::is_same<Real, float>::value) return t - S.sub_v;
            else return S.coef * t - S.sub_v;
        }
        return S.coef * t;
    }
    if (S.kind == 2) {
        if (j == S.js) return t + S.add_js;
        if (j == S.v) return S.drop ? Real(0) : t - S.sub_v;
    }
    return t;
}



// Double-float values hi + lo (|lo| <= ulp(hi)/2) for the atom weights of the
// active-set kernels: a pairwise step adds and subtracts the same amount, and
// in this representation it does so exactly enough that a row's mass does not
// drift over many thousands of steps. Round-to-nearest intrinsics throughout
// (never contracted or reordered).
struct DF {
    float hi, lo;
};
__device__ inline DF df_norm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return DF{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ inline DF df_add(DF x, DF y) {
    const float s = __fadd_rn(x.hi, y.hi);
    const float bb = __fsub_rn(s, x.hi);
    float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    return df_norm(s, e);
}
__device__ inline DF df_mulf(DF x, float c) {
    const float p = __fmul_rn(x.hi, c);
    float e = __fmaf_rn(x.hi, c, -p);
    e = __fmaf_rn(x.lo, c, e);
    return df_norm(p, e);
}

// Exact product x * y of two floats as a double-float (TwoProduct).
__device__ inline DF df_prod(float x, float y) {
    const float p = __fmul_rn(x, y);
    return DF{p, __fmaf_rn(x, y, -p)};
}

// New weight of atom column j under step S (the atom-list form of apply()).
// The convex-combination steps are evaluated as t - gamma t (+ gamma a_i at
// j*) and t + gamma t (- gamma a_i at v), with gamma a_i an exact product, so
// that the rounding of 1 -/+ gamma never enters: the row's mass changes by
// gamma (a_i - sum t) + O(eps^2), as it does in exact arithmetic (where it is
// 0). ai is the row weight; mv is the mass a pairwise step moves (the whole
// away atom on a drop step).
__device__ inline DF apply_atom(const Step<float> &S, int j, DF t, DF mv, float ai) {
    if (S.kind == 0) {
        const DF gt = df_mulf(t, S.gamma);
        DF r = df_add(t, DF{-gt.hi, -gt.lo});
        if (j == S.js) r = df_add(r, df_prod(S.gamma, ai));
        return r;
    }
    if (S.kind == 1) {
        if (j == S.v && S.drop) return DF{0.f, 0.f};
        DF r = df_add(t, df_mulf(t, S.gamma));
        if (j == S.v) {
            const DF ga = df_prod(S.gamma, ai);
            r = df_add(r, DF{-ga.hi, -ga.lo});
        }
        return r;
    }
    if (S.kind == 2) {
        if (j == S.js) return df_add(t, mv);
        if (j == S.v) return S.drop ? DF{0.f, 0.f} : df_add(t, DF{-mv.hi, -mv.lo});
    }
    return t;
}

// Row quantities the control warp of the active-set kernels gathers over the
// atoms before the LMO vertex is known. With gmax the largest gradient over
// the active atoms (away vertex v):
//   g_aw = sum_k t_k (gmax - g_k) >= 0            (away-direction decrease)
//   s2   = sum_k t_k^2,  dda = ||t - a e_v||^2    (sums of squares)
// Because the atom weights sum to a_i, the FW gap follows without the
// cancellation of sum t g - a gmin:  g_fw = a (gmax - gmin) - g_aw.
struct AtomStats {
    float gmax, g_aw, s2, dda, t_v;
    int v, nnz;
    int vpos;  // position of v in the atom record (-1 if none)
};

// Decision of one block update from the atom statistics (Alg. 1 / A.2 with
// the line search of eq. 8 / eq. 10; pairwise steps are decided separately).
__device__ inline Step<float> decide_atoms(const AtomStats &A, float gmin, int js, float t_js, float ai,
                                           int variant, int step, float rho, int m, long long k) {
    Step<float> S;
    S.kind = -1; S.gamma = 0.f; S.js = js; S.v = A.v;
    S.coef = 1.f; S.add_js = 0.f; S.sub_v = 0.f; S.drop = false;
    if (!(ai > 0.f)) return S;
    const float g_fw = ai * (A.gmax - gmin) - A.g_aw;
    const bool fw = variant == SR_OT_BCFW || A.nnz <= 1 || g_fw >= A.g_aw || !(A.t_v < ai);
    if (fw) {
        float gam;
        if (variant == SR_OT_BCFW && step == SR_OT_DEC) {
            gam = (float)((2.0 * (double)m) / ((double)k + 2.0 * (double)m));
        } else {
            const float dd = (A.s2 - t_js * t_js) + (ai - t_js) * (ai - t_js);
            gam = line_search<float>(g_fw, dd > 0.f ? dd : 0.f, rho, 1.f);
        }
        S.kind = 0; S.gamma = gam; S.coef = 1.f - gam; S.add_js = gam * ai;
        return S;
    }
    const float alpha = A.t_v / ai;
    const float gmx = alpha / (1.f - alpha);
    const float gam = line_search<float>(A.g_aw, A.dda, rho, gmx);
    S.kind = 1; S.gamma = gam; S.coef = 1.f + gam; S.sub_v = gam * ai;
    S.drop = gam >= gmx;
    return S;
}

}  // namespace srot
