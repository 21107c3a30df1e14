// internal.h -- launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace srot {

// Cost source of one instance.
enum CostMode : int {
    kCostGiven = 0,  // dense C (m x n) in device memory
    kCostPts3 = 1,   // points X (m x 3), Y (n x 3): C_ij = ||x_i - y_j||^2 on the fly
};

// Device-side layout of one certificate (Thm 2) result: doubles.
enum CertSlot : int {
    kCertF = 0,      // objective f(T)
    kCertG = 1,      // linearisation gap g(T)
    kCertW = 2,      // Lagrangian dual w(T) = f - g
    kCertLin = 3,    // <C, T>
    kCertPen = 4,    // (rho/2) ||T^T 1 - b||^2
    kCertRel = 5,    // g / f
    kCertStop = 6,   // 1.0 when g <= tol * f and the plan is feasible
    kCertFeas = 7,   // max_i |sum_j T_ij - a_i| / a_i (row-sum defect)
    kCertCount = 8
};

// One instance as seen by the certificate and solver kernels.
template <typename Real>
struct Inst {
    int m, n;
    int cost_mode;
    const Real *C;   // kCostGiven
    const Real *X;   // kCostPts3
    const Real *Y;
    const Real *a;
    const Real *b;
};

// A plan counts as feasible for the stopping test when every row sum is
// within this relative distance of a_i (FP32 plans drift by rounding).
constexpr double kFeasTol = 1e-5;

// Workspace the certificate needs (all device pointers).
struct CertWork {
    double *partial;     // nchunks * n
    int nchunks, rows_per_chunk;
    double *r64;         // n: exact residual s - b
    float *rq32;         // n: (float)(rho * r) for the FP32 argmin
    double *colpart;     // per-block partials of the column pass (2 per block)
    int ncolblocks;
    double *rowpart;     // per-block partials of the row pass (3 per block: <C,T>, sum a min, max defect)
    int nrowblocks;
    double *cert;        // kCertCount doubles
};

// Sizes of the certificate workspace for an m x n instance.
void cert_work_shape(int m, int n, int *nchunks, int *rows_per_chunk, int *ncolblocks,
                     int *nrowblocks);

// Certificate of plan T (Thm 2). If refresh_q is non-null, the solver's
// running residual is overwritten from the exact column sums: the FP32 path
// keeps q = rho * r, the FP64 path keeps r (both in double). g_rows
// (optional) receives per-row gaps, js_out (optional) each row's LMO vertex.
template <typename Real>
void launch_certificate(const Inst<Real> &in, const Real *T, double rho, double tol,
                        const CertWork &w, double *refresh_q, double *g_rows, cudaStream_t st,
                        int *js_out = nullptr);

// T = (a_i e_0) (Thm 1) and the solver's initial residual (FP32: q = rho (T^T1 - b);
// FP64: r = T^T1 - b with the column sums taken in ascending row order).
template <typename Real>
void launch_init_plan(const Inst<Real> &in, Real *T, int warm, double rho, double *q,
                      cudaStream_t st);

// Exact column-sum residual for the solver (ascending row order, FP64 accumulate).
template <typename Real>
void launch_init_residual(const Inst<Real> &in, const Real *T, double rho, double *q,
                          cudaStream_t st);

// Uniform random permutation of 0..m-1 for epoch `epoch` (sort by splitmix64 keys).
void launch_make_perm(unsigned long long seed, long long epoch, int m, int *perm,
                      uint64_t *keybuf, int *idxbuf, cudaStream_t st);
size_t make_perm_scratch_bytes(int m);

// BF16 tensor-core cost C = |x~|^2 + |y~|^2 - 2 X~ Y~^T (X~, Y~: BF16-rounded
// points; FP32 accumulation and norms). ws: cost_bf16_workspace(m, n, d)
// bytes; err_dev: an int set to 1 if a bounded wait gave up. Returns an error
// message for unsupported arguments (nothing launched), else nullptr.
size_t cost_bf16_workspace(int m, int n, int d);
const char *launch_cost_bf16(int m, int n, int d, const float *X, const float *Y, float *C, void *ws,
                             int *err_dev, cudaStream_t st);

// Materialise C_ij = ||x_i - y_j||^2 (euclid: ||x_i - y_j||_2) for any d on
// the CUDA cores, summed over ascending k without contraction.
template <typename Real>
void launch_cost_plain(int m, int n, int d, const Real *X, const Real *Y, Real *C,
                       cudaStream_t st, bool euclid = false);

// Single-instance epoch of block updates.
template <typename Real>
struct EpochArgs {
    Inst<Real> in;
    Real *T;
    double *q;               // running residual: FP32 path rho * r, FP64 path r
    double rho;
    int variant, step, order;
    long long k0;            // block updates before this epoch
    long long epoch;
    unsigned long long seed;
    const int *perm;         // order == PERMUTE
    double *g_store;         // order == GAP_ADAPTIVE: per-row gaps (m)
    int ga_inner;            // 1: recompute g_i after each update
    int *trace;
    long long trace_cap;
    int *status;
    bool vec;                // T (and C) rows start on 16-byte boundaries
    int4 *atoms;             // sparse kernel: per-row atom records (m x kAtomRecord)
    int *resume;             // sparse kernel: set to the update index where it stopped
    const int *resume_in;    // dense kernel: start at *resume_in, or return if it is < 0
    int *sticky;             // active-set kernels: set when a row outgrows its record; once set, they
                             // leave every later epoch to the dense kernel (*resume = 0)
    long long spin_limit;    // speculative kernel: probes before a wait gives up (0: default)
    const int *gate;         // speculative kernel: wait for *gate != 0 before the first update
    const float *C32;        // FP64 single-warp kernel: the FP32 rounding of C (argmin screen)
};

// Gap-adaptive epoch (Alg. A.4): rows drawn with probability proportional to
// max(g_i, 0) from A.g_store; A.ga_inner re-evaluates g_i after each update.
// False if m or n is too large.
template <typename Real>
bool launch_epoch_ga(const EpochArgs<Real> &args, cudaStream_t st);
int epoch_ga_max_m();

// Full Frank-Wolfe step (Alg. A.1) after a certificate that wrote every
// row's LMO vertex js: exact line search (step == ELS, gap g read from
// cert[kCertG]) or the decay 2 / (it + 2), then T <- (1 - gamma) T + gamma S.
// upart: workspace of fw_upart_size(n) doubles; gamma_dev: one double.
int fw_upart_size(int n);
template <typename Real>
void launch_fw_step(const Inst<Real> &in, Real *T, const int *js, const double *r64,
                    const double *cert, int step, long long it, double rho, double *upart,
                    double *gamma_dev, cudaStream_t st);

// Atom record of one row for the active-set kernels: entry 0 = {count, 0, 0,
// 0}, then up to 63 entries {column, weight hi bits, weight lo bits, 0}
// (double-float weights); 1 KiB.
constexpr int kAtomRecord = 64;

// Sparse-support epoch (FP32, away / pairwise steps). False if n is too large.
bool launch_epoch_sparse(const EpochArgs<float> &args, cudaStream_t st);
// Pipelined sparse-support epoch for pairwise steps (the next row's argmin
// overlaps the current update). False unless BCPFW and n fits.
bool launch_epoch_pipe(const EpochArgs<float> &args, cudaStream_t st);
// Speculative pairwise epoch: the LMOs of the next rows are taken ahead
// against an older residual and repaired at the columns changed since. chain:
// 1 or 3 chain warps in rotation, or kSpecChainSplit (two preparer warps and
// one decider). False unless BCPFW, d = 3 points, cyclic or permuted order
// and n <= 4096.
constexpr int kSpecChainSplit = 0;
bool launch_epoch_spec(const EpochArgs<float> &args, cudaStream_t st, int chain);

// FP64 BCFW epoch on one warp (n <= epoch_f64w_max_n(), cost given as C):
// false if the arguments are outside what it takes.
bool launch_epoch_f64w(const EpochArgs<double> &args, cudaStream_t st);
int epoch_f64w_max_n();
// C32[e] = fl32(C[e]) for the single-warp kernel's argmin screen.
void launch_round_cost(const double *C, float *C32, size_t count, cudaStream_t st);

// Atom records of a dense plan; *overflow becomes 1 if a row has > 63 atoms.
void launch_build_atoms(int m, int n, const float *T, int4 *rec, int *overflow, cudaStream_t st);

// Returns false when n exceeds the single-instance kernel's limit.
template <typename Real>
bool launch_epoch(const EpochArgs<Real> &args, cudaStream_t st);

int epoch_max_n(bool fp64);

// The speculative kernel's chain alone (chain_warps 1 or 3), `updates` times;
// *status is set to kDevTimeout if a wait gave up; sink: one float.
void launch_chain_floor(int chain_warps, int updates, int *status, float *sink, cudaStream_t st);

// Message returned by sr_ot_last_error(NULL) on this thread (errors of calls
// that have no handle).
void set_handleless_error(const char *msg);

// ---- adjoint (envelope-theorem gradients) ---------------------------------
// One instance of an adjoint launch. Offsets are in elements; dX, dY and db
// use the offsets of X, Y and b.
struct AdjInst {
    int m, n;
    long long oX, oY, ob, oT, oa;
    int nbands, rh, ncol;  // row bands of rh rows; column tiles of 256 x (16 / element size)
    int tile0;             // first tile (CTA) of this instance
    long long col0, row0;  // prefix sums of n and m over the instances
    long long ocp, orp;    // offsets of the column / row partials
    int fin0;              // first block of this instance in the finishing pass
};

struct AdjTotals {
    long long tiles, cols, rows, colpart, rowpart, fin_blocks;
};

template <typename Real>
struct AdjArgs {
    const AdjInst *inst;
    int ninst, d;
    double rho;
    const Real *X, *Y, *b, *T;
    Real *dC, *dX, *dY, *db;  // any may be null (dC only for one instance)
    Real *colpart, *rowpart;  // workspace from adj_plan's totals
    // colour-transfer tail (any may be null): barycentric projection (m x d,
    // offsets of X), row weights a (offsets oa), per-finishing-block squared
    // marginal errors (total_fin doubles), zero entries of T per instance,
    // and per instance {||T1 - a||, ||T^T 1 - b||, e_c, sparsity}
    Real *xhat;
    const Real *a;
    double *tpart;
    unsigned long long *zeros;
    double *tstats;
    int total_tiles;
    long long total_cols, total_rows;
    int total_fin;  // blocks of the finishing pass
};

// ---- evaluation metrics against a reference plan (Sec. 5, v and vi) ------
template <typename Real>
struct LpMetricsArgs {
    int m, n;
    const Real *T, *L;  // the plan and the reference plan T*_LP
    const Real *C;      // given cost, or null: d = 3 points X, Y
    const Real *X, *Y;
    bool euclid;        // points: the Euclidean cost instead of the squared one
};
// Blocks of the metrics pass (4 doubles of partial sums each).
int lp_metrics_blocks(int m);
// out[0..3] = sum (t - l)^2, sum l^2, <T, C>, <L, C>; part: 4 doubles per block.
template <typename Real>
void launch_lp_metrics(const LpMetricsArgs<Real> &A, double *part, double *out, cudaStream_t st);

// Padded width of the per-entry partial vector (x or y, then 1): 4, 8, 16 or 32.
int adj_width(int d);
// Tiles and workspace of a set of instances (elem_bytes: 4 or 8); fills
// out[k] except the offsets oX, oY, ob, oT.
AdjTotals adj_plan(int ninst, const int *m, const int *n, int d, int elem_bytes, AdjInst *out);
// Launch the tile pass and the finishing pass (and, with tstats, the
// transfer statistics); false if d is out of range.
template <typename Real>
bool launch_adjoint(const AdjArgs<Real> &A, cudaStream_t st);

}  // namespace srot
