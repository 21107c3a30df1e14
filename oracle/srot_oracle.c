/*
 * srot_oracle.c -- plain, slow, FP64 CPU oracle for block-coordinate
 * Frank-Wolfe on the squared-l2 semi-relaxed optimal transport problem
 * (Fukunaga & Kasai, "Fast block-coordinate Frank-Wolfe algorithm for
 * semi-relaxed optimal transport", arXiv 2103.05857).
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only callers. This file shares no
 * code, header, table or helper with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Orientation. The paper makes the COLUMNS of T the blocks (T^T 1_m = b is
 * exact, T 1_n ~ a is penalised with weight 1/(2 lambda)). This file uses
 * the transposed orientation throughout: T is m x n row-major, ROW i is the
 * block t_i in a_i * Delta_n (T 1_n = a exactly), and the column sums
 * s = T^T 1_m are pulled toward b by (rho/2) ||s - b||^2, rho = 1/lambda.
 *
 *   f(T)      = <C, T> + (rho/2) ||r||^2,  r = T^T 1_m - b      (Sec. 3, eq. 5)
 *   grad_i    = C_{i,:} + rho * r                                 (Sec. 3.1)
 *   LMO       = a_i e_{j*}, j* = argmin_j grad_ij                 (Sec. 3.1, eq. 7)
 *   g_i       = <t_i - a_i e_{j*}, grad_i>                        (Sec. 4.2, eq. 11)
 *   g(T)      = sum_i g_i                                         (Thm 2)
 *   w(T)      = f - sum_i <t_i, grad_i> + sum_i a_i min_j grad_ij (Thm 2, App. D)
 *
 * Parity status of each function is recorded in the test suite: every
 * function below is pinned by at least one check that does not re-type its
 * formula (KKT brute force, closed forms, vertex enumeration, finite
 * differences of f, deterministic FW rate).
 *
 * Arithmetic. Compiled with -ffp-contract=off: every product and sum below
 * is one IEEE-754 rounding, in the order written. Sums run in ascending
 * index order. Nothing is blocked, fused or reordered.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Random numbers: splitmix64 (Steele, Lea & Flood, OOPSLA 2014). The k-th
 * output (k >= 1) of a generator seeded with z0 is mix(z0 + k * GOLDEN).
 * Streams are separated by xoring a stream id into the top byte of the seed.
 * ------------------------------------------------------------------------- */
#define OR_GOLDEN 0x9E3779B97F4A7C15ULL

static uint64_t or_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t srot_or_draw(uint64_t seed, uint64_t stream, uint64_t counter) {
    uint64_t z0 = seed ^ (stream << 56);
    return or_mix(z0 + (counter + 1ULL) * OR_GOLDEN);
}

/* floor(u * m) for a 64-bit uniform u, as the high word of the 128-bit
 * product (no modulo bias beyond 2^-64). */
static int or_scale(uint64_t u, int m) {
    unsigned __int128 p = (unsigned __int128)u * (unsigned __int128)(uint64_t)m;
    return (int)(uint64_t)(p >> 64);
}

/* ---------------------------------------------------------------------------
 * Cost: C_ij = ||x_i - y_j||_2^2 (squared Euclidean), summed over the
 * feature axis in ascending order. The paper's colour experiments use the
 * non-squared distance (Sec. 5.1); the squared cost is this library's
 * workload and is selected by `squared` = 1 (0 takes the square root).
 * ------------------------------------------------------------------------- */
void srot_or_cost(int m, int n, int d, const double *X, const double *Y,
                  int squared, double *C) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k) {
                double dl = X[(size_t)i * d + k] - Y[(size_t)j * d + k];
                acc = acc + dl * dl;
            }
            C[(size_t)i * n + j] = squared ? acc : sqrt(acc);
        }
}

/* ---------------------------------------------------------------------------
 * Certificate at a fixed plan T (Thm 2): objective f, linearisation gap g,
 * Lagrangian dual value w, per-row gaps g_rows (optional) and column sums s
 * (optional). out[0] = f, out[1] = g, out[2] = w, out[3] = <C,T>,
 * out[4] = (rho/2)||r||^2.
 * ------------------------------------------------------------------------- */
void srot_or_certificate(int m, int n, const double *C, const double *a,
                         const double *b, double rho, const double *T,
                         double *out, double *g_rows, double *s_out) {
    double *s = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; ++j) s[j] = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) s[j] = s[j] + T[(size_t)i * n + j];
    for (int j = 0; j < n; ++j) r[j] = s[j] - b[j];

    double lin = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) lin = lin + C[(size_t)i * n + j] * T[(size_t)i * n + j];
    double rr = 0.0;
    for (int j = 0; j < n; ++j) rr = rr + r[j] * r[j];
    double pen = 0.5 * rho * rr;
    double f = lin + pen;

    double g = 0.0, sum_tg = 0.0, sum_amin = 0.0;
    for (int i = 0; i < m; ++i) {
        double gmin = 0.0, tg = 0.0;
        for (int j = 0; j < n; ++j) {
            double gr = C[(size_t)i * n + j] + rho * r[j];
            if (j == 0 || gr < gmin) gmin = gr;
            tg = tg + T[(size_t)i * n + j] * gr;
        }
        double gi = (n > 0) ? tg - a[i] * gmin : 0.0;
        if (g_rows) g_rows[i] = gi;
        g = g + gi;
        sum_tg = sum_tg + tg;
        if (n > 0) sum_amin = sum_amin + a[i] * gmin;
    }
    out[0] = f;
    out[1] = g;
    out[2] = f - sum_tg + sum_amin;
    out[3] = lin;
    out[4] = pen;
    if (s_out)
        for (int j = 0; j < n; ++j) s_out[j] = s[j];
    free(s);
    free(r);
}

/* ---------------------------------------------------------------------------
 * Solver options (mirrors the library's option set in meaning, not in code).
 * ------------------------------------------------------------------------- */
enum { OR_BCFW = 0, OR_BCAFW = 1, OR_BCPFW = 2, OR_FW = 3 };
enum { OR_CYCLIC = 0, OR_PERMUTE = 1, OR_UNIFORM = 2, OR_GAP = 3 };
enum { OR_DEC = 0, OR_ELS = 1 };

typedef struct {
    int variant;          /* OR_BCFW / OR_BCAFW / OR_BCPFW / OR_FW            */
    int order;            /* block order (ignored by OR_FW)                  */
    int step;             /* OR_DEC or OR_ELS                                */
    int gap_every;        /* certificate every this many epochs (>= 1)       */
    double rho;           /* penalty weight, rho = 1/lambda_paper, >= 0      */
    double tol_rel_gap;   /* stop when g <= tol * f (0: run max_epochs)      */
    long long max_epochs; /* epochs (FW: iterations)                         */
    int ga_M;             /* GA: global update every ga_M epochs             */
    int ga_global_only;   /* GA: 1 = no inner update (GAS)                   */
    double ga_init_const; /* GA: 0 = exact g_i at start, >0 = this constant  */
    uint64_t seed;
    int warm_start;       /* 1: T holds a feasible start; 0: T0 = a_i e_0    */
} srot_or_opts;

typedef struct {
    double f, g, w;
    long long epochs, updates;
    long long n_hist; /* certificate records written to hist */
    int converged;
    int status; /* 0 ok, -1 invalid options */
} srot_or_result;

/* Exact line search on a quadratic along d (Sec. 3.1 eq. 8, Sec. 4.1 eq. 10):
 * minimise phi(gamma) = -num*gamma + (rho/2) dd gamma^2 over [0, gmax]. */
static double or_line_search(double num, double dd, double rho, double gmax) {
    if (!(num > 0.0)) return 0.0;
    double den = rho * dd;
    if (!(den > 0.0)) return gmax;
    double gam = num / den;
    return gam < gmax ? gam : gmax;
}

/* Row gap g_i at the current T and r (Sec. 4.2 eq. 11). */
static double or_row_gap(int n, const double *Ci, const double *ti, double ai,
                         const double *r, double rho) {
    double gmin = 0.0, tg = 0.0;
    for (int j = 0; j < n; ++j) {
        double gr = Ci[j] + rho * r[j];
        if (j == 0 || gr < gmin) gmin = gr;
        tg = tg + ti[j] * gr;
    }
    return tg - ai * gmin;
}

typedef struct {
    int jstar;   /* LMO vertex (Sec. 3.1 eq. 7)                       */
    int v;       /* away vertex (-1 if unused)                         */
    int dir;     /* 0 FW, 1 away, 2 pairwise, -1 no move               */
    double gamma;
} or_step_info;

/* Apply one decided block update to row t_i and the residual r (Alg. 1,
 * line "t_i <- (1 - gamma) t_i + gamma s_i"; Alg. A.2 away step; Alg. A.3
 * pairwise step, with the atom v dropped when gamma reaches its maximum).
 * dir: 0 Frank-Wolfe direction toward a_i e_js, 1 away direction from the
 * atom v (gamma_max = alpha_v / (1 - alpha_v), alpha_v = t_iv / a_i),
 * 2 pairwise move of mass from v to js (gamma_max = alpha_v), -1 no move. */
static void or_apply_step(int n, double *ti, double ai, double *r, int dir, int js,
                          int v, double gam) {
    if (dir == 0) {
        double omg = 1.0 - gam;
        for (int j = 0; j < n; ++j) {
            double told = ti[j];
            double tnew = omg * told;
            if (j == js) tnew = tnew + gam * ai;
            r[j] = r[j] + (tnew - told);
            ti[j] = tnew;
        }
    } else if (dir == 1) {
        double alpha = ti[v] / ai;
        double gmax = alpha / (1.0 - alpha);
        double opg = 1.0 + gam;
        for (int j = 0; j < n; ++j) {
            double told = ti[j];
            double tnew = opg * told;
            if (j == v) tnew = (gam >= gmax) ? 0.0 : tnew - gam * ai;
            r[j] = r[j] + (tnew - told);
            ti[j] = tnew;
        }
    } else if (dir == 2 && v != js) {
        double gmax = ti[v] / ai;
        double moved = (gam >= gmax) ? ti[v] : gam * ai;
        double tv_old = ti[v], tj_old = ti[js];
        double tv_new = (gam >= gmax) ? 0.0 : tv_old - moved;
        double tj_new = tj_old + moved;
        r[v] = r[v] + (tv_new - tv_old);
        r[js] = r[js] + (tj_new - tj_old);
        ti[v] = tv_new;
        ti[js] = tj_new;
    }
}

/* One block update of row i (Alg. 1; Alg. A.2; Alg. A.3). `k` is the
 * global block-update counter used by the decay rule 2m/(k+2m) (Alg. 1,
 * written for m blocks). T row i and r are updated in place. */
static int or_block_update(int m, int n, const double *Ci, double *ti, double ai,
                           double *r, double *grad, const srot_or_opts *o,
                           long long k, or_step_info *info) {
    const double rho = o->rho;
    info->jstar = -1; info->v = -1; info->dir = -1; info->gamma = 0.0;
    if (n <= 0) return 0;

    for (int j = 0; j < n; ++j) grad[j] = Ci[j] + rho * r[j];
    int js = 0;
    for (int j = 1; j < n; ++j)
        if (grad[j] < grad[js]) js = j;
    info->jstar = js;
    if (!(ai > 0.0)) return 0; /* empty block: nothing to move */

    double dot = 0.0;
    for (int j = 0; j < n; ++j) dot = dot + ti[j] * grad[j];
    double g_fw = dot - ai * grad[js];

    if (o->variant == OR_BCFW) {
        double gam;
        if (o->step == OR_DEC) {
            gam = (2.0 * (double)m) / ((double)k + 2.0 * (double)m);
        } else {
            double dd = 0.0;
            for (int j = 0; j < n; ++j) {
                double dl = ti[j] - (j == js ? ai : 0.0);
                dd = dd + dl * dl;
            }
            gam = or_line_search(g_fw, dd, rho, 1.0);
        }
        or_apply_step(n, ti, ai, r, 0, js, -1, gam);
        info->dir = 0; info->gamma = gam;
        return 0;
    }

    if (o->step != OR_ELS) return -1; /* away/pairwise steps need the line search */

    /* away vertex: argmax of grad over the active atoms {j : t_ij > 0}. */
    int v = -1, nnz = 0;
    for (int j = 0; j < n; ++j)
        if (ti[j] > 0.0) {
            ++nnz;
            if (v < 0 || grad[j] > grad[v]) v = j;
        }
    info->v = v;
    if (v < 0) return 0;

    if (o->variant == OR_BCAFW) {
        double g_aw = ai * grad[v] - dot;
        if (nnz == 1 || g_fw >= g_aw) {
            double dd = 0.0;
            for (int j = 0; j < n; ++j) {
                double dl = ti[j] - (j == js ? ai : 0.0);
                dd = dd + dl * dl;
            }
            double gam = or_line_search(g_fw, dd, rho, 1.0);
            or_apply_step(n, ti, ai, r, 0, js, v, gam);
            info->dir = 0; info->gamma = gam;
        } else {
            double alpha = ti[v] / ai;
            double gmax = alpha / (1.0 - alpha);
            double dd = 0.0;
            for (int j = 0; j < n; ++j) {
                double dl = ti[j] - (j == v ? ai : 0.0);
                dd = dd + dl * dl;
            }
            double gam = or_line_search(g_aw, dd, rho, gmax);
            or_apply_step(n, ti, ai, r, 1, js, v, gam);
            info->dir = 1; info->gamma = gam;
        }
        return 0;
    }

    /* OR_BCPFW: move mass from the away atom v to the FW vertex j*. */
    if (v == js) { info->dir = 2; info->gamma = 0.0; return 0; }
    double g_pw = ai * (grad[v] - grad[js]);
    double dd = 2.0 * ai * ai;
    double gmax = ti[v] / ai;
    double gam = or_line_search(g_pw, dd, rho, gmax);
    or_apply_step(n, ti, ai, r, 2, js, v, gam);
    info->dir = 2; info->gamma = gam;
    return 0;
}

/* Public single-step entry for the line-search and step-rule pins: applies one
 * block update of row i to (T, r) and reports (jstar, v, dir, gamma). */
int srot_or_block_step(int m, int n, const double *C, const double *a, double *T,
                       double *r, int i, long long k, const srot_or_opts *o,
                       int *jstar, int *v, int *dir, double *gamma) {
    double *grad = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    or_step_info info;
    int st = or_block_update(m, n, C + (size_t)i * n, T + (size_t)i * n, a[i], r,
                             grad, o, k, &info);
    free(grad);
    *jstar = info.jstar; *v = info.v; *dir = info.dir; *gamma = info.gamma;
    return st;
}

/* Public entry that applies a GIVEN decision (direction dir, LMO vertex
 * jstar, away atom v, step gamma) to row i of (T, r) with the same update
 * arithmetic as a block step; used to follow another solver's decision at a
 * point where the two may legitimately differ (an exact tie). */
void srot_or_apply_step(int n, const double *a, double *T, double *r, int i, int dir,
                        int jstar, int v, double gamma) {
    or_apply_step(n, T + (size_t)i * n, a[i], r, dir, jstar, v, gamma);
}

/* Uniform permutation of 0..m-1 for epoch e: positions sorted by a random
 * 64-bit key per index (ties by index). */
typedef struct { uint64_t key; int idx; } or_keyed;
static int or_cmp_keyed(const void *x, const void *y) {
    const or_keyed *p = (const or_keyed *)x, *q = (const or_keyed *)y;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}
void srot_or_permutation(uint64_t seed, long long epoch, int m, int *perm) {
    or_keyed *kv = (or_keyed *)malloc(sizeof(or_keyed) * (size_t)(m > 0 ? m : 1));
    for (int t = 0; t < m; ++t) {
        kv[t].key = srot_or_draw(seed, 1, (uint64_t)epoch * (uint64_t)m + (uint64_t)t);
        kv[t].idx = t;
    }
    qsort(kv, (size_t)m, sizeof(or_keyed), or_cmp_keyed);
    for (int t = 0; t < m; ++t) perm[t] = kv[t].idx;
    free(kv);
}

/* Gap-adaptive sampling (Sec. 4.2, Alg. A.4): index i with probability
 * proportional to max(g_i, 0), by inverse transform of one uniform draw u64:
 * with u = top 53 bits of u64 in [0, 1) and cum_i the running sum of the
 * clamped gaps, the smallest i of positive weight with cum_i > u * total
 * (a linear scan of the cumulative sum). All weights zero: uniform index. */
int srot_or_sample_from(const double *gst, int m, uint64_t u64) {
    double total = 0.0;
    for (int i = 0; i < m; ++i) total = total + (gst[i] > 0.0 ? gst[i] : 0.0);
    if (!(total > 0.0)) return or_scale(u64, m);
    double u = (double)(u64 >> 11) * 0x1.0p-53;
    double target = u * total;
    double cum = 0.0;
    int last_pos = 0;
    for (int i = 0; i < m; ++i) {
        double w = gst[i] > 0.0 ? gst[i] : 0.0;
        if (w > 0.0) last_pos = i;
        cum = cum + w;
        if (cum > target && w > 0.0) return i;
    }
    return last_pos;
}

/* Uniform block index floor(u * m) of draw u64 (the uniform order, Sec. 3.1). */
int srot_or_uniform_index(uint64_t u64, int m) { return or_scale(u64, m); }

static int or_sample_gap(const double *gst, int m, uint64_t seed, long long k) {
    return srot_or_sample_from(gst, m, srot_or_draw(seed, 3, (uint64_t)k));
}

static void or_global_gap_update(int m, int n, const double *C, const double *a,
                                 const double *T, const double *r, double rho,
                                 double *gst) {
    for (int i = 0; i < m; ++i)
        gst[i] = or_row_gap(n, C + (size_t)i * n, T + (size_t)i * n, a[i], r, rho);
}

/* ---------------------------------------------------------------------------
 * Block-coordinate solvers: BCFW (Alg. 1), BCAFW (Alg. A.2), BCPFW
 * (Alg. A.3), each with cyclic / permuted / uniform / gap-adaptive (Alg. A.4)
 * block order. One epoch is m block updates. The certificate (Thm 2) is taken
 * every `gap_every` epochs and at the last epoch; the solve stops when
 * g <= tol_rel_gap * f.
 *
 * trace_i / trace_j (optional, capacity trace_cap) receive, per update, the
 * block index and the LMO vertex j*. hist (optional, capacity 3 * max_epochs)
 * receives (epoch, f, g) for each certificate taken.
 * ------------------------------------------------------------------------- */
static int or_solve_fw(int m, int n, const double *C, const double *a,
                       const double *b, const srot_or_opts *o, double *T,
                       double *hist, srot_or_result *res);

int srot_or_solve_ex(int m, int n, const double *C, const double *a, const double *b,
                     const srot_or_opts *o, double *T, int *trace_i, int *trace_j,
                     long long trace_cap, double *hist, double *ga_hist, double *T_hist,
                     srot_or_result *res);

int srot_or_solve(int m, int n, const double *C, const double *a, const double *b,
                  const srot_or_opts *o, double *T, int *trace_i, int *trace_j,
                  long long trace_cap, double *hist, srot_or_result *res) {
    return srot_or_solve_ex(m, n, C, a, b, o, T, trace_i, trace_j, trace_cap, hist, NULL, NULL, res);
}

/* As srot_or_solve, and optionally records, at the end of every epoch e
 * (after that epoch's global gap update, if one is due): the sampling gaps
 * g_i into ga_hist[e*m .. e*m+m) (gap-adaptive order only) and the plan into
 * T_hist[e*m*n .. (e+1)*m*n). Both need max_epochs epochs of room. */
int srot_or_solve_ex(int m, int n, const double *C, const double *a, const double *b,
                     const srot_or_opts *o, double *T, int *trace_i, int *trace_j,
                     long long trace_cap, double *hist, double *ga_hist, double *T_hist,
                     srot_or_result *res) {
    memset(res, 0, sizeof(*res));
    if (m <= 0 || n <= 0 || o->gap_every < 1 || o->rho < 0.0) { res->status = -1; return -1; }
    if (o->variant != OR_BCFW && o->variant != OR_FW && o->step != OR_ELS) { res->status = -1; return -1; }
    if (o->variant == OR_FW) return or_solve_fw(m, n, C, a, b, o, T, hist, res);

    size_t mn = (size_t)m * (size_t)n;
    if (!o->warm_start) {
        for (size_t e = 0; e < mn; ++e) T[e] = 0.0;
        for (int i = 0; i < m; ++i) T[(size_t)i * n] = a[i];
    }
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *grad = (double *)malloc(sizeof(double) * (size_t)n);
    int *perm = (int *)malloc(sizeof(int) * (size_t)m);
    double *gst = (double *)malloc(sizeof(double) * (size_t)m);
    for (int j = 0; j < n; ++j) r[j] = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) r[j] = r[j] + T[(size_t)i * n + j];
    for (int j = 0; j < n; ++j) r[j] = r[j] - b[j];

    const int ga = (o->order == OR_GAP);
    const int gaM = o->ga_global_only ? 1 : (o->ga_M > 0 ? o->ga_M : 1);
    if (ga) {
        if (o->ga_init_const > 0.0)
            for (int i = 0; i < m; ++i) gst[i] = o->ga_init_const;
        else
            or_global_gap_update(m, n, C, a, T, r, o->rho, gst);
    }

    long long k = 0;
    long long nh = 0;
    int status = 0;
    double cert[5] = {0, 0, 0, 0, 0};
    for (long long ep = 0; ep < o->max_epochs; ++ep) {
        if (o->order == OR_PERMUTE) srot_or_permutation(o->seed, ep, m, perm);
        for (int p = 0; p < m; ++p) {
            int i;
            if (o->order == OR_CYCLIC) i = p;
            else if (o->order == OR_PERMUTE) i = perm[p];
            else if (o->order == OR_UNIFORM) i = or_scale(srot_or_draw(o->seed, 2, (uint64_t)k), m);
            else i = or_sample_gap(gst, m, o->seed, k);
            or_step_info info;
            int st = or_block_update(m, n, C + (size_t)i * n, T + (size_t)i * n, a[i], r,
                                     grad, o, k, &info);
            if (st) { status = st; break; }
            if (ga && !o->ga_global_only)
                gst[i] = or_row_gap(n, C + (size_t)i * n, T + (size_t)i * n, a[i], r, o->rho);
            if (trace_i && k < trace_cap) { trace_i[k] = i; trace_j[k] = info.jstar; }
            ++k;
        }
        if (status) break;
        if (ga && ((ep + 1) % gaM == 0)) or_global_gap_update(m, n, C, a, T, r, o->rho, gst);
        if (ga && ga_hist)
            for (int i = 0; i < m; ++i) ga_hist[(size_t)ep * m + i] = gst[i];
        if (T_hist)
            for (size_t e = 0; e < mn; ++e) T_hist[(size_t)ep * mn + e] = T[e];
        int last = (ep + 1 == o->max_epochs);
        if ((ep + 1) % o->gap_every == 0 || last) {
            srot_or_certificate(m, n, C, a, b, o->rho, T, cert, NULL, NULL);
            if (hist) { hist[3 * nh] = (double)(ep + 1); hist[3 * nh + 1] = cert[0]; hist[3 * nh + 2] = cert[1]; }
            ++nh;
            res->epochs = ep + 1;
            if (o->tol_rel_gap > 0.0 && cert[1] <= o->tol_rel_gap * cert[0]) { res->converged = 1; break; }
        }
    }
    if (o->max_epochs <= 0) srot_or_certificate(m, n, C, a, b, o->rho, T, cert, NULL, NULL);
    res->f = cert[0]; res->g = cert[1]; res->w = cert[2];
    res->updates = k;
    res->n_hist = nh;
    res->status = status;
    free(r); free(grad); free(perm); free(gst);
    return status;
}

/* Full Frank-Wolfe (Alg. A.1): every block's LMO at the same T, then one
 * global step, decay 2/(k+2) or the exact line search stated with Alg. A.1. The gap
 * computed for the step is the certificate of the current T (Thm 2). */
static int or_solve_fw(int m, int n, const double *C, const double *a,
                       const double *b, const srot_or_opts *o, double *T,
                       double *hist, srot_or_result *res) {
    size_t mn = (size_t)m * (size_t)n;
    if (!o->warm_start) {
        for (size_t e = 0; e < mn; ++e) T[e] = 0.0;
        for (int i = 0; i < m; ++i) T[(size_t)i * n] = a[i];
    }
    const double rho = o->rho;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    int *js = (int *)malloc(sizeof(int) * (size_t)m);
    double cert[5];
    long long it = 0;
    for (it = 0; it < o->max_epochs; ++it) {
        for (int j = 0; j < n; ++j) r[j] = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) r[j] = r[j] + T[(size_t)i * n + j];
        for (int j = 0; j < n; ++j) r[j] = r[j] - b[j];
        double g = 0.0;
        for (int i = 0; i < m; ++i) {
            const double *Ci = C + (size_t)i * n;
            const double *ti = T + (size_t)i * n;
            int jb = 0;
            double gb = Ci[0] + rho * r[0];
            double tg = 0.0;
            for (int j = 0; j < n; ++j) {
                double gr = Ci[j] + rho * r[j];
                if (gr < gb) { gb = gr; jb = j; }
                tg = tg + ti[j] * gr;
            }
            js[i] = jb;
            g = g + (tg - a[i] * gb);
        }
        srot_or_certificate(m, n, C, a, b, rho, T, cert, NULL, NULL);
        if (hist) { hist[3 * it] = (double)it; hist[3 * it + 1] = cert[0]; hist[3 * it + 2] = g; }
        res->n_hist = it + 1;
        if (o->tol_rel_gap > 0.0 && g <= o->tol_rel_gap * cert[0]) { res->converged = 1; break; }
        double gam;
        if (o->step == OR_DEC) {
            gam = 2.0 / ((double)it + 2.0);
        } else {
            /* u = (T - S)^T 1: column sums of T minus those of S. */
            for (int j = 0; j < n; ++j) u[j] = 0.0;
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < n; ++j) u[j] = u[j] + T[(size_t)i * n + j];
            for (int i = 0; i < m; ++i) u[js[i]] = u[js[i]] - a[i];
            double uu = 0.0;
            for (int j = 0; j < n; ++j) uu = uu + u[j] * u[j];
            gam = or_line_search(g, uu, rho, 1.0);
        }
        double omg = 1.0 - gam;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double t = omg * T[(size_t)i * n + j];
                if (j == js[i]) t = t + gam * a[i];
                T[(size_t)i * n + j] = t;
            }
    }
    srot_or_certificate(m, n, C, a, b, rho, T, cert, NULL, NULL);
    res->f = cert[0]; res->g = cert[1]; res->w = cert[2];
    res->epochs = it; res->updates = it * (long long)m;
    res->status = 0;
    free(r); free(u); free(js);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Envelope-theorem gradients of the optimal value at a plan T for the
 * squared-Euclidean point cost C_ij = ||x_i - y_j||^2:
 *   d/dC = T,
 *   dX   = 2 (diag(T 1_n) X - T Y),
 *   dY   = 2 (diag(T^T 1_m) Y - T^T X),
 *   db   = -rho (T^T 1_m - b).
 * Not in the paper; it follows from differentiating f at fixed optimal T.
 * Any output may be NULL.
 * ------------------------------------------------------------------------- */
void srot_or_adjoint(int m, int n, int d, const double *X, const double *Y,
                     const double *b, double rho, const double *T, double *dX,
                     double *dY, double *db) {
    if (dX)
        for (int i = 0; i < m; ++i) {
            double rs = 0.0;
            for (int j = 0; j < n; ++j) rs = rs + T[(size_t)i * n + j];
            for (int k = 0; k < d; ++k) {
                double ty = 0.0;
                for (int j = 0; j < n; ++j) ty = ty + T[(size_t)i * n + j] * Y[(size_t)j * d + k];
                dX[(size_t)i * d + k] = 2.0 * (rs * X[(size_t)i * d + k] - ty);
            }
        }
    if (dY || db) {
        double *s = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        for (int j = 0; j < n; ++j) s[j] = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) s[j] = s[j] + T[(size_t)i * n + j];
        if (dY)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < d; ++k) {
                    double tx = 0.0;
                    for (int i = 0; i < m; ++i) tx = tx + T[(size_t)i * n + j] * X[(size_t)i * d + k];
                    dY[(size_t)j * d + k] = 2.0 * (s[j] * Y[(size_t)j * d + k] - tx);
                }
        if (db)
            for (int j = 0; j < n; ++j) db[j] = -rho * (s[j] - b[j]);
        free(s);
    }
}
